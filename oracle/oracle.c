/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the SpGEMM /
 * SpRef / SpAsgn path (Buluc & Gilbert, "Parallel Sparse Matrix-Matrix
 * Multiplication and Indexing: Implementation and Experiments").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path: the semiring and type codes below are this file's own.
 *
 * Conventions: 0-based indices (the paper is 1-based, Section 2), CSR with
 * int64 row offsets and int32 column ids, rows strictly increasing in column.
 *
 * Built with -O2 -ffp-contract=off so that no multiply-add is fused: every
 * product and every sum is one IEEE-754 operation in the order written here.
 * An OpenMP pragma splits independent rows across threads for timing only;
 * each row is computed exactly as in the serial loop.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* semirings (Section 1: SpGEMM over any semiring) */
#define O_PLUS_TIMES 0 /* (+, x)                                        */
#define O_OR_AND 1     /* (or, and): structure only                     */
#define O_MIN_PLUS 2   /* (min, +)                                      */
#define O_SELECT2ND 3  /* mul(a,b) = b: left operand is a 0/1 selector  */
#define O_SELECT1ST 4  /* mul(a,b) = a: right operand is a 0/1 selector */

/* value types */
#define O_F64 0
#define O_F32 1
#define O_I32 2
#define O_I64 3
#define O_BOOL 4

/* status codes */
#define O_OK 0
#define O_EINVAL -1
#define O_ESELECT -2   /* a selector product had two contributions to one entry */
#define O_EOVERFLOW -3 /* (min,+) int32 sum out of range                          */
#define O_ENOMEM -4

typedef struct {
  int64_t m, n;
  const int64_t *p; /* row offsets, m+1      */
  const int32_t *j; /* column ids            */
  const void *v;    /* values or NULL (bool) */
  int32_t t;        /* value type            */
} ocsr;

static double getd(const void *v, int t, int64_t q) {
  switch (t) {
    case O_F64: return ((const double *)v)[q];
    case O_F32: return (double)((const float *)v)[q];
    case O_I32: return (double)((const int32_t *)v)[q];
    case O_I64: return (double)((const int64_t *)v)[q];
  }
  return 1.0;
}

/* ------------------------------------------------------------------ flops --
 * flops(A.B) = number of nonzero multiplications (Section 2 notation):
 * sum over stored A(i,k) of nnz(B(k,:)).  Per-row counts for rows [r0,r1). */
int64_t oracle_flops(const ocsr *A, const ocsr *B, int64_t r0, int64_t r1, int64_t *rowflops) {
  int64_t total = 0;
  for (int64_t i = r0; i < r1; ++i) {
    int64_t f = 0;
    for (int64_t q = A->p[i]; q < A->p[i + 1]; ++q) {
      int64_t k = A->j[q];
      f += B->p[k + 1] - B->p[k];
    }
    if (rowflops) rowflops[i - r0] = f;
    total += f;
  }
  return total;
}

/* ----------------------------------------------------------- symbolic SpGEMM --
 * Row-wise Gustavson (Algorithm 1 applied to rows: C(i,:) += A(i,k) * B(k,:)
 * for every stored A(i,k)), with the dense sparse accumulator of Figure 1
 * reduced to its occupancy part: mark[j] holds the last row that touched
 * column j.  Returns nnz(C(r0:r1,:)); rownnz[i-r0] gets each row's count. */
int64_t oracle_spgemm_symbolic(const ocsr *A, const ocsr *B, int64_t r0, int64_t r1,
                               int64_t *rownnz, int nthreads) {
  int64_t total = 0;
  int failed = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : total)
  {
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(B->n > 0 ? B->n : 1));
    if (!mark) {
#pragma omp atomic write
      failed = 1;
    } else {
      for (int64_t c = 0; c < B->n; ++c) mark[c] = -1;
#pragma omp for schedule(dynamic, 64)
      for (int64_t i = r0; i < r1; ++i) {
        int64_t cnt = 0;
        for (int64_t q = A->p[i]; q < A->p[i + 1]; ++q) {
          int64_t k = A->j[q];
          for (int64_t s = B->p[k]; s < B->p[k + 1]; ++s) {
            int32_t c = B->j[s];
            if (mark[c] != i) {
              mark[c] = i;
              ++cnt;
            }
          }
        }
        rownnz[i - r0] = cnt;
        total += cnt;
      }
      free(mark);
    }
  }
  return failed ? O_ENOMEM : total;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------ numeric SpGEMM --
 * The same row-wise Gustavson pass with the full SPA of Figure 1: a dense
 * value array, the occupancy stamps and the list of touched columns.
 * For each row i, k runs over A(i,:) in stored order and j over B(k,:) in
 * stored order; the first product reaching column j initialises the SPA
 * entry and every later one is combined with the semiring's add, so the
 * additive identity is never used.  The touched list is then sorted and the
 * row is emitted in ascending column order.
 *
 * Accumulation precision: (+,x) on f64 adds in double; (+,x) on f32 forms
 * each product in double (exact for two floats) and sums in double, rounding
 * once to float when the entry is emitted; (+,x) on i64 wraps modulo 2^64;
 * (min,+) on f32 forms a+b in float (the paper's semiring on floats) and keeps
 * the minimum; (min,+) on i32 forms a+b in 64 bits and fails if it leaves the
 * int32 range.
 *
 * bound (may be NULL): per output entry, sum over contributions of |a|*|b| in
 * double, the scale of the floating-point tolerance.
 *
 * cp: r1-r0+1 output offsets relative to the first row (from the symbolic pass).
 * cv: output values of the result type (NULL for (or,and)).                   */
int oracle_spgemm_numeric(int sr, const ocsr *A, const ocsr *B, int64_t r0, int64_t r1,
                          const int64_t *cp, int32_t *cj, void *cv, double *bound, int nthreads) {
  int status = O_OK;
  int ot; /* output value type */
  if (sr == O_OR_AND) ot = O_BOOL;
  else if (sr == O_SELECT2ND) ot = B->t;
  else if (sr == O_SELECT1ST) ot = A->t;
  else {
    if (A->t != B->t) return O_EINVAL;
    ot = A->t;
  }
  if (sr == O_PLUS_TIMES && !(ot == O_F64 || ot == O_F32 || ot == O_I64)) return O_EINVAL;
  if (sr == O_MIN_PLUS && !(ot == O_F32 || ot == O_I32)) return O_EINVAL;

#pragma omp parallel num_threads(nthreads)
  {
    size_t n = (size_t)(B->n > 0 ? B->n : 1);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * n);
    double *accd = (double *)malloc(sizeof(double) * n);   /* f64 / f32 sums      */
    float *accf = (float *)malloc(sizeof(float) * n);      /* (min,+) f32         */
    int64_t *acci = (int64_t *)malloc(sizeof(int64_t) * n); /* integer semirings  */
    double *bnd = (double *)malloc(sizeof(double) * n);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!mark || !accd || !accf || !acci || !bnd || !touched) {
#pragma omp atomic write
      status = O_ENOMEM;
    } else {
      for (size_t c = 0; c < n; ++c) mark[c] = -1;
#pragma omp for schedule(dynamic, 64)
      for (int64_t i = r0; i < r1; ++i) {
        int64_t nt = 0;
        for (int64_t q = A->p[i]; q < A->p[i + 1]; ++q) {
          int64_t k = A->j[q];
          for (int64_t s = B->p[k]; s < B->p[k + 1]; ++s) {
            int32_t c = B->j[s];
            int first = (mark[c] != i);
            if (first) {
              mark[c] = i;
              touched[nt++] = c;
            }
            switch (sr) {
              case O_OR_AND:
                break;
              case O_PLUS_TIMES:
                if (ot == O_I64) {
                  uint64_t prod = (uint64_t)((const int64_t *)A->v)[q] *
                                  (uint64_t)((const int64_t *)B->v)[s];
                  acci[c] = first ? (int64_t)prod : (int64_t)((uint64_t)acci[c] + prod);
                } else {
                  double a = getd(A->v, A->t, q), b = getd(B->v, B->t, s);
                  double prod = a * b;
                  accd[c] = first ? prod : accd[c] + prod;
                  double mag = fabs(a) * fabs(b);
                  bnd[c] = first ? mag : bnd[c] + mag;
                }
                break;
              case O_MIN_PLUS:
                if (ot == O_F32) {
                  float sum = ((const float *)A->v)[q] + ((const float *)B->v)[s];
                  accf[c] = (first || sum < accf[c]) ? sum : accf[c];
                } else {
                  int64_t sum = (int64_t)((const int32_t *)A->v)[q] + (int64_t)((const int32_t *)B->v)[s];
                  if (sum > INT32_MAX || sum < INT32_MIN) {
#pragma omp atomic write
                    status = O_EOVERFLOW;
                  }
                  acci[c] = (first || sum < acci[c]) ? sum : acci[c];
                }
                break;
              case O_SELECT2ND:
              case O_SELECT1ST: {
                /* exactly one contribution per output entry is the operator's precondition */
                if (!first) {
#pragma omp atomic write
                  status = O_ESELECT;
                }
                const void *src = (sr == O_SELECT2ND) ? B->v : A->v;
                int64_t at = (sr == O_SELECT2ND) ? s : q;
                if (ot == O_F64) accd[c] = ((const double *)src)[at];
                else if (ot == O_F32) accf[c] = ((const float *)src)[at];
                else if (ot == O_I32) acci[c] = ((const int32_t *)src)[at];
                else if (ot == O_I64) acci[c] = ((const int64_t *)src)[at];
                break;
              }
            }
          }
        }
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        int64_t base = cp[i - r0];
        if (cp[i - r0 + 1] - base != nt) {
#pragma omp atomic write
          status = O_EINVAL;
          continue;
        }
        for (int64_t t = 0; t < nt; ++t) {
          int32_t c = touched[t];
          cj[base + t] = c;
          if (bound) bound[base + t] = (sr == O_PLUS_TIMES && ot != O_I64) ? bnd[c] : 0.0;
          if (ot == O_BOOL) continue;
          int sel = (sr == O_SELECT2ND || sr == O_SELECT1ST);
          switch (ot) {
            case O_F64: ((double *)cv)[base + t] = accd[c]; break;
            case O_F32:
              ((float *)cv)[base + t] = (sr == O_PLUS_TIMES) ? (float)accd[c] : accf[c];
              break;
            case O_I32: ((int32_t *)cv)[base + t] = (int32_t)acci[c]; break;
            case O_I64: ((int64_t *)cv)[base + t] = acci[c]; break;
          }
          (void)sel;
        }
      }
    }
    free(mark); free(accd); free(accf); free(acci); free(bnd); free(touched);
  }
  return status;
}

/* ------------------------------------------------------------------ SpRef --
 * B = A(I,J) (Section 3): row t of B is row I[t] of A, and column p of B is
 * column J[p] of A, in the order the indices are given; repeated indices
 * repeat rows/columns.  Computed directly by index, not through products:
 * pos lists, for every column k of A, the positions p with J[p] == k in
 * increasing p; entry (I[t],k,v) of A yields (t,p,v) for each p in pos(k).
 * Each output row is then sorted by p.
 * Two calls: count (cp == NULL: fills rownnz, returns nnz(B)) and fill.      */
typedef struct {
  int32_t p;
  int64_t src; /* index of the A entry supplying the value */
} pv_t;

static int cmp_pv(const void *a, const void *b) {
  int32_t x = ((const pv_t *)a)->p, y = ((const pv_t *)b)->p;
  return (x > y) - (x < y);
}

static size_t tsize(int t) {
  switch (t) {
    case O_F64: case O_I64: return 8;
    case O_F32: case O_I32: return 4;
  }
  return 0;
}

int64_t oracle_spref(const ocsr *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ,
                     int64_t *rownnz, const int64_t *cp, int32_t *cj, void *cv) {
  for (int64_t t = 0; t < nI; ++t)
    if (I[t] < 0 || I[t] >= A->m) return O_EINVAL;
  for (int64_t p = 0; p < nJ; ++p)
    if (J[p] < 0 || J[p] >= A->n) return O_EINVAL;
  /* pos(k) as CSR: posp[k]..posp[k+1] in posv, increasing p */
  int64_t *posp = (int64_t *)calloc((size_t)A->n + 1, sizeof(int64_t));
  int32_t *posv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nJ > 0 ? nJ : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(A->n > 0 ? A->n : 1));
  if (!posp || !posv || !fill) { free(posp); free(posv); free(fill); return O_ENOMEM; }
  for (int64_t p = 0; p < nJ; ++p) posp[J[p] + 1]++;
  for (int64_t k = 0; k < A->n; ++k) posp[k + 1] += posp[k];
  for (int64_t k = 0; k < A->n; ++k) fill[k] = posp[k];
  for (int64_t p = 0; p < nJ; ++p) posv[fill[J[p]]++] = (int32_t)p;

  int64_t total = 0;
  size_t es = tsize(A->t);
  for (int64_t t = 0; t < nI; ++t) {
    int64_t r = I[t], cnt = 0;
    for (int64_t q = A->p[r]; q < A->p[r + 1]; ++q) cnt += posp[A->j[q] + 1] - posp[A->j[q]];
    if (!cp) {
      rownnz[t] = cnt;
      total += cnt;
      continue;
    }
    pv_t *tmp = (pv_t *)malloc(sizeof(pv_t) * (size_t)(cnt > 0 ? cnt : 1));
    int64_t w = 0;
    for (int64_t q = A->p[r]; q < A->p[r + 1]; ++q) {
      int64_t k = A->j[q];
      for (int64_t s = posp[k]; s < posp[k + 1]; ++s) {
        tmp[w].p = posv[s];
        tmp[w].src = q;
        ++w;
      }
    }
    qsort(tmp, (size_t)cnt, sizeof(pv_t), cmp_pv);
    int64_t base = cp[t];
    for (int64_t e = 0; e < cnt; ++e) {
      cj[base + e] = tmp[e].p;
      if (es) memcpy((char *)cv + (size_t)(base + e) * es, (const char *)A->v + (size_t)tmp[e].src * es, es);
    }
    total += cnt;
    free(tmp);
  }
  free(posp); free(posv); free(fill);
  return total;
}

/* ----------------------------------------------------------------- SpAsgn --
 * C = A with A(I,J) replaced by B (Section 3.1): C = A + R*B*Q - S*A*T, with
 * the subtraction read as an elementwise product of A with the structural
 * negation of S*A*T (no additive inverse is assumed).  Computed directly by
 * index: rpos[r] = q if I[q] == r else -1, cpos[c] = q if J[q] == c else -1.
 * Row r of C is a copy of A(r,:) when rpos[r] < 0; otherwise it keeps the
 * entries (c,v) of A(r,:) with cpos[c] < 0 and adds (J[q], w) for every
 * (q,w) in B(rpos[r],:), in ascending column order.
 * accumulate = 1 gives Liu's extend-add A(I,J) = A(I,J) + B: entries of A in
 * the block are kept and combined with B's through the semiring add
 * (sr = O_PLUS_TIMES or O_MIN_PLUS; O_OR_AND for structure only).
 * I and J must be duplicate-free (returns O_EINVAL otherwise).
 * Two calls: count (cp == NULL) and fill.                                    */
typedef struct {
  int32_t c;
  int32_t from_b;  /* 0: A, 1: B */
  int64_t src;
} cv_t;

static int cmp_cv(const void *a, const void *b) {
  const cv_t *x = (const cv_t *)a, *y = (const cv_t *)b;
  if (x->c != y->c) return (x->c > y->c) - (x->c < y->c);
  return (x->from_b > y->from_b) - (x->from_b < y->from_b);
}

int64_t oracle_spasgn(const ocsr *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ,
                      const ocsr *B, int accumulate, int sr,
                      int64_t *rownnz, const int64_t *cp, int32_t *cj, void *cv) {
  if (B->m != nI || B->n != nJ) return O_EINVAL;
  if (A->t != B->t) return O_EINVAL;
  int32_t *rpos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->m > 0 ? A->m : 1));
  int32_t *cpos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(A->n > 0 ? A->n : 1));
  if (!rpos || !cpos) { free(rpos); free(cpos); return O_ENOMEM; }
  for (int64_t r = 0; r < A->m; ++r) rpos[r] = -1;
  for (int64_t c = 0; c < A->n; ++c) cpos[c] = -1;
  int64_t status = 0;
  for (int64_t q = 0; q < nI && !status; ++q) {
    if (I[q] < 0 || I[q] >= A->m || rpos[I[q]] >= 0) status = O_EINVAL;
    else rpos[I[q]] = (int32_t)q;
  }
  for (int64_t q = 0; q < nJ && !status; ++q) {
    if (J[q] < 0 || J[q] >= A->n || cpos[J[q]] >= 0) status = O_EINVAL;
    else cpos[J[q]] = (int32_t)q;
  }
  if (status) { free(rpos); free(cpos); return status; }

  size_t es = tsize(A->t);
  int64_t total = 0;
  for (int64_t r = 0; r < A->m; ++r) {
    int64_t na = A->p[r + 1] - A->p[r];
    if (rpos[r] < 0) {
      if (!cp) { rownnz[r] = na; total += na; continue; }
      int64_t base = cp[r];
      for (int64_t e = 0; e < na; ++e) {
        cj[base + e] = A->j[A->p[r] + e];
        if (es) memcpy((char *)cv + (size_t)(base + e) * es, (const char *)A->v + (size_t)(A->p[r] + e) * es, es);
      }
      total += na;
      continue;
    }
    int64_t br = rpos[r];
    int64_t nb = B->p[br + 1] - B->p[br];
    cv_t *tmp = (cv_t *)malloc(sizeof(cv_t) * (size_t)(na + nb > 0 ? na + nb : 1));
    int64_t w = 0;
    for (int64_t q = A->p[r]; q < A->p[r + 1]; ++q) {
      if (!accumulate && cpos[A->j[q]] >= 0) continue; /* structurally negated block */
      tmp[w].c = A->j[q]; tmp[w].from_b = 0; tmp[w].src = q; ++w;
    }
    for (int64_t q = B->p[br]; q < B->p[br + 1]; ++q) {
      tmp[w].c = J[B->j[q]]; tmp[w].from_b = 1; tmp[w].src = q; ++w;
    }
    qsort(tmp, (size_t)w, sizeof(cv_t), cmp_cv);
    /* merge equal columns (only possible with accumulate: one from A, one from B) */
    int64_t out = 0;
    for (int64_t e = 0; e < w; ++e) {
      int merge = (e > 0 && tmp[e].c == tmp[e - 1].c);
      if (!merge) ++out;
      if (!cp) continue;
      int64_t at = cp[r] + out - 1;
      if (!merge) {
        cj[at] = tmp[e].c;
        const void *src = tmp[e].from_b ? B->v : A->v;
        if (es) memcpy((char *)cv + (size_t)at * es, (const char *)src + (size_t)tmp[e].src * es, es);
        continue;
      }
      /* tmp[e-1] is A's entry, tmp[e] is B's: combine with the semiring add */
      int64_t qa = tmp[e - 1].src, qb = tmp[e].src;
      switch (A->t) {
        case O_F64: {
          double a = ((const double *)A->v)[qa], b = ((const double *)B->v)[qb];
          ((double *)cv)[at] = (sr == O_MIN_PLUS) ? (b < a ? b : a) : a + b;
          break;
        }
        case O_F32: {
          float a = ((const float *)A->v)[qa], b = ((const float *)B->v)[qb];
          ((float *)cv)[at] = (sr == O_MIN_PLUS) ? (b < a ? b : a) : a + b;
          break;
        }
        case O_I32: {
          int32_t a = ((const int32_t *)A->v)[qa], b = ((const int32_t *)B->v)[qb];
          ((int32_t *)cv)[at] = (sr == O_MIN_PLUS) ? (b < a ? b : a) : (int32_t)((uint32_t)a + (uint32_t)b);
          break;
        }
        case O_I64: {
          int64_t a = ((const int64_t *)A->v)[qa], b = ((const int64_t *)B->v)[qb];
          ((int64_t *)cv)[at] = (sr == O_MIN_PLUS) ? (b < a ? b : a) : (int64_t)((uint64_t)a + (uint64_t)b);
          break;
        }
        default: break;
      }
    }
    if (!cp) rownnz[r] = out;
    total += out;
    free(tmp);
  }
  free(rpos); free(cpos);
  return total;
}

/* ----------------------------------------------------------------- sparse --
 * C = sparse(i, j, v, m, n) in the notation of Section 2: the m x n matrix
 * whose entry (i(k), j(k)) holds v(k), k = 0..nnz-1.  Several tuples may name
 * one position; they are then combined with the semiring's add, taken in
 * increasing k: the sum (O_PLUS_TIMES; F64, F32, I64), the minimum
 * (O_MIN_PLUS; F32, I32) or the logical or (O_OR_AND; O_BOOL, v unused).
 * Floating-point sums are formed in double and rounded once to the value
 * type; integer sums wrap modulo 2^64.  bound (optional) receives, per entry
 * of C, the sum of |v(k)| over its tuples: the scale of the rounding error of
 * a sum formed in the value type in any order.
 * Called twice: with cp == NULL it fills rownnz[m] and returns nnz(C); then,
 * with cp the scanned offsets, it fills cj, cv and bound.                   */
typedef struct {
  int32_t i, j;
  int64_t k;
} ijk_t;

static int cmp_ijk(const void *a, const void *b) {
  const ijk_t *x = (const ijk_t *)a, *y = (const ijk_t *)b;
  if (x->i != y->i) return (x->i > y->i) - (x->i < y->i);
  if (x->j != y->j) return (x->j > y->j) - (x->j < y->j);
  return (x->k > y->k) - (x->k < y->k);
}

int64_t oracle_sparse(const int32_t *I, const int32_t *J, const void *V, int64_t nnz, int64_t m,
                      int64_t n, int t, int sr, int64_t *rownnz, const int64_t *cp, int32_t *cj,
                      void *cv, double *bound) {
  int ok = (sr == O_PLUS_TIMES && (t == O_F64 || t == O_F32 || t == O_I64)) ||
           (sr == O_MIN_PLUS && (t == O_F32 || t == O_I32)) || (sr == O_OR_AND && t == O_BOOL);
  if (!ok || nnz < 0 || m < 0 || n < 0 || (t != O_BOOL && nnz > 0 && !V)) return O_EINVAL;
  for (int64_t k = 0; k < nnz; ++k)
    if (I[k] < 0 || I[k] >= m || J[k] < 0 || J[k] >= n) return O_EINVAL;
  ijk_t *s = (ijk_t *)malloc(sizeof(ijk_t) * (size_t)(nnz > 0 ? nnz : 1));
  if (!s) return O_ENOMEM;
  for (int64_t k = 0; k < nnz; ++k) { s[k].i = I[k]; s[k].j = J[k]; s[k].k = k; }
  qsort(s, (size_t)nnz, sizeof(ijk_t), cmp_ijk);
  if (!cp)
    for (int64_t r = 0; r < m; ++r) rownnz[r] = 0;
  int64_t out = 0;
  for (int64_t e = 0; e < nnz;) {
    int64_t f = e + 1; /* tuples e..f-1 share one position */
    while (f < nnz && s[f].i == s[e].i && s[f].j == s[e].j) ++f;
    if (!cp) {
      ++rownnz[s[e].i];
    } else {
      /* rows are visited in increasing order, so entry `out` is the next slot */
      cj[out] = s[e].j;
      double sa = 0.0;
      for (int64_t q = e; q < f; ++q) sa += fabs(getd(V, t, s[q].k));
      if (bound) bound[out] = (t == O_BOOL) ? 0.0 : sa;
      switch (t) {
        case O_F64: case O_F32: {
          double acc = getd(V, t, s[e].k);
          for (int64_t q = e + 1; q < f; ++q) {
            double x = getd(V, t, s[q].k);
            acc = (sr == O_MIN_PLUS) ? (x < acc ? x : acc) : acc + x;
          }
          if (t == O_F64) ((double *)cv)[out] = acc;
          else ((float *)cv)[out] = (float)acc;
          break;
        }
        case O_I32: {
          int32_t acc = ((const int32_t *)V)[s[e].k];
          for (int64_t q = e + 1; q < f; ++q) {
            int32_t x = ((const int32_t *)V)[s[q].k];
            acc = x < acc ? x : acc;
          }
          ((int32_t *)cv)[out] = acc;
          break;
        }
        case O_I64: {
          uint64_t acc = (uint64_t)((const int64_t *)V)[s[e].k];
          for (int64_t q = e + 1; q < f; ++q) acc += (uint64_t)((const int64_t *)V)[s[q].k];
          ((int64_t *)cv)[out] = (int64_t)acc;
          break;
        }
        default: break;
      }
    }
    ++out;
    e = f;
  }
  free(s);
  return out;
}

/* ------------------------------------------------------------- DCSC / DCSR --
 * Doubly compressed form (Section 2.2): drop the repeated pointers of empty
 * columns (rows) and keep the ids of the non-empty ones in JC, parallel to
 * CP.  Works on either orientation: given a compressed-pointer array ptr of
 * length dim+1, writes jc[nz] and cp[nz+1] and returns nz.                   */
int64_t oracle_doubly_compress(const int64_t *ptr, int64_t dim, int64_t *jc, int64_t *cp) {
  int64_t nz = 0;
  for (int64_t c = 0; c < dim; ++c) {
    if (ptr[c + 1] > ptr[c]) {
      if (jc) jc[nz] = c;
      if (cp) cp[nz] = ptr[c];
      ++nz;
    }
  }
  if (cp) cp[nz] = ptr[dim];
  return nz;
}
