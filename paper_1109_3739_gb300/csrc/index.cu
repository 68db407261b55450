// index.cu -- device pieces of SpRef and SpAsgn (Section 3.1).
//
// The selection matrices of the SpRef and SpAsgn listings are built on the
// device in CSR form (the constructor sparse(i, j, 1, m, n) for their
// special shapes):
//   SpRef  R = sparse(1:len(I), I, 1, len(I), m)  -> row t holds column I[t]
//          Q = sparse(J, 1:len(J), 1, n, len(J))  -> row k holds every p with
//                                                    J[p] == k, increasing
//   SpAsgn R = sparse(I, 1:mb, 1, ma, mb)         -> row I[q] holds column q
//          Q = sparse(1:nb, J, 1, nb, na)         -> row q holds column J[q]
// and the final step of SpAsgn, the elementwise product of A with the
// structural negation of S*A*T plus R*B*Q: an entry (r, c) of A is in the
// structure of S*A*T exactly when r is in I and c is in J, so the negation is
// applied through the inverse index maps rpos/cpos, so neither S*A*T nor its
// negation is ever materialised (Section 3.1).
#include "common.cuh"
#include "internal.h"

namespace hs {

static int grid1(int64_t n, int nt = 256) {
  int64_t g = (n + nt - 1) / nt;
  int64_t cap = (int64_t)sm_count() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_iota_i64(int64_t *p, int64_t n) { GRID_STRIDE(i, n) p[i] = i; }

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) { GRID_STRIDE(i, n) a[i] = v; }
void launch_fill_i32(int32_t *a, int64_t n, int32_t v, cudaStream_t st) {
  if (n > 0) {
    count_launch();
    k_fill_i32<<<grid1(n), 256, 0, st>>>(a, n, v);
  }
}

__global__ void k_iota_i32(int32_t *p, int64_t n) { GRID_STRIDE(i, n) p[i] = (int32_t)i; }
void launch_iota_i32(int32_t *p, int64_t n, cudaStream_t st) {
  if (n > 0) {
    count_launch();
    k_iota_i32<<<grid1(n), 256, 0, st>>>(p, n);
  }
}

// Q of SpRef: counts per row k go to Qp[k+1]; indices outside [0, bound)
// are skipped (the host reports them), so this may run before the range check
__global__ void k_count_idx(const int32_t *X, int64_t n, int64_t bound, int64_t *cnt) {
  GRID_STRIDE(i, n) {
    const int32_t x = X[i];
    if (x >= 0 && x < bound) atomicAdd(reinterpret_cast<unsigned long long *>(cnt + x + 1), 1ull);
  }
}
void launch_build_Q_count(const int32_t *J, int64_t nJ, int64_t bound, int64_t *Qp_counts, cudaStream_t st) {
  if (nJ > 0) {
    count_launch();
    k_count_idx<<<grid1(nJ), 256, 0, st>>>(J, nJ, bound, Qp_counts);
  }
}
// the largest of n counts, into *out (zeroed by the caller)
__global__ void k_max_count(const int64_t *cnt, int64_t n, unsigned long long *out) {
  unsigned long long mx = 0;
  GRID_STRIDE(i, n) mx = max(mx, (unsigned long long)cnt[i]);
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}
void launch_max_count(const int64_t *cnt, int64_t n, unsigned long long *out, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  k_max_count<<<grid1(n), 256, 0, st>>>(cnt, n, out);
}

// Q of SpRef: cur holds the row offsets on entry and is advanced by atomics;
// rows are then put in increasing order of p by an insertion sort, used only
// when no row holds more than 32 entries (one per repetition of k in J)
__global__ void k_fill_idx(const int32_t *X, int64_t n, int64_t *cur, int32_t *out) {
  GRID_STRIDE(i, n) {
    const unsigned long long at = atomicAdd(reinterpret_cast<unsigned long long *>(cur + X[i]), 1ull);
    out[at] = (int32_t)i;
  }
}
__global__ void k_sort_short_rows(const int64_t *ptr, int32_t *j, int64_t rows) {
  GRID_STRIDE(r, rows) {
    const int64_t b = ptr[r], e = ptr[r + 1];
    for (int64_t x = b + 1; x < e; ++x) {
      const int32_t v = j[x];
      int64_t y = x - 1;
      while (y >= b && j[y] > v) {
        j[y + 1] = j[y];
        --y;
      }
      j[y + 1] = v;
    }
  }
}
// Qcur: a copy of the finished offsets (length n+1); Qj is sorted per row
// using the offsets that precede Qcur in the caller's layout (Qcur - (n+1))
void launch_build_Q_fill(const int32_t *J, int64_t nJ, int64_t *Qcur, int32_t *Qj, cudaStream_t st) {
  if (nJ > 0) {
    count_launch();
    k_fill_idx<<<grid1(nJ), 256, 0, st>>>(J, nJ, Qcur, Qj);
  }
}
void launch_sort_short_rows(const int64_t *ptr, int32_t *j, int64_t rows, cudaStream_t st) {
  if (rows > 0) {
    count_launch();
    k_sort_short_rows<<<grid1(rows), 256, 0, st>>>(ptr, j, rows);
  }
}

// ----------------------------------------------------- SpRef by gathering
// B = A(I, J) without forming R*A: the rows I[t] of A are laid end to end
// (gathered entry g of output row t is entry A.p[I[t]] + g - G[t] of A,
// G the scanned row lengths), every gathered entry (t, c, v) becomes one
// tuple (t, p, v) for each p with J[p] == c (Q's row c), and the tuples are
// sorted by (t, p) -- or, when J is strictly increasing, written in place,
// already in order.

// G[t + 1] = length of row I[t] (G[0] is zero)
__global__ void k_gather_len(const int64_t *Ap, const int32_t *I, int64_t nI, int64_t *G) {
  GRID_STRIDE(t, nI) G[t + 1] = Ap[I[t] + 1] - Ap[I[t]];
}
// inc[G[t]] += 1 for every row starting inside [0, total): after an
// inclusive scan, inc[g] - 1 is the output row of gathered entry g
__global__ void k_row_starts(const int64_t *G, int64_t nI, int64_t total, int64_t *inc) {
  GRID_STRIDE(t, nI) {
    const int64_t g = G[t];
    if (g < total) atomicAdd(reinterpret_cast<unsigned long long *>(inc + g), 1ull);
  }
}
__device__ __forceinline__ void gather_entry(const GatherArgs &a, int64_t g, int64_t &t, int64_t &q, int &c) {
  t = a.row[g] - 1;
  q = a.Ap[a.I[t]] + (g - a.G[t]);
  c = a.Aj[q];
}
// W[g] = number of tuples entry g makes (|{p : J[p] == c}|)
__global__ void k_gather_w(GatherArgs a, int64_t *W) {
  GRID_STRIDE(g, a.total) {
    int64_t t, q;
    int c;
    gather_entry(a, g, t, q, c);
    W[g] = (c >= 0 && c < a.ncols) ? a.Qp[c + 1] - a.Qp[c] : 0;
  }
}
__device__ __forceinline__ void copy_val(void *dst, int64_t at, const void *src, int64_t q, int vb) {
  if (vb == 8) reinterpret_cast<uint64_t *>(dst)[at] = reinterpret_cast<const uint64_t *>(src)[q];
  else if (vb == 4) reinterpret_cast<uint32_t *>(dst)[at] = reinterpret_cast<const uint32_t *>(src)[q];
}
// the tuples, entry g's at [W[g-1], W[g]) of the scanned counts
__global__ void k_gather_fill(GatherArgs a, const int64_t *W, int32_t *ti, int32_t *pj, void *tv) {
  GRID_STRIDE(g, a.total) {
    int64_t t, q;
    int c;
    gather_entry(a, g, t, q, c);
    int64_t at = g > 0 ? W[g - 1] : 0;
    if (at == W[g]) continue;  // no tuple (and c may be any id)
    for (int64_t k = a.Qp[c]; k < a.Qp[c + 1]; ++k, ++at) {
      ti[at] = (int32_t)t;
      pj[at] = a.Qj[k];
      copy_val(tv, at, a.Av, q, a.vb);
    }
  }
}
// J strictly increasing: each entry makes at most one tuple and a row's
// tuples come out in increasing p, so they are B's entries as they stand
__global__ void k_gather_direct(GatherArgs a, const int64_t *W, int32_t *Bj, void *Bv) {
  GRID_STRIDE(g, a.total) {
    const int64_t before = g > 0 ? W[g - 1] : 0;
    if (W[g] == before) continue;
    int64_t t, q;
    int c;
    gather_entry(a, g, t, q, c);
    Bj[before] = a.Qj[a.Qp[c]];
    copy_val(Bv, before, a.Av, q, a.vb);
  }
}
// B's offsets from the scanned tuple counts: Bp[t] = W[G[t] - 1]
__global__ void k_gather_offsets(const int64_t *G, int64_t nI, const int64_t *W, int64_t *Bp) {
  GRID_STRIDE(t, nI + 1) {
    const int64_t g = G[t];
    Bp[t] = g > 0 ? W[g - 1] : 0;
  }
}
// flag bit 4: J not strictly increasing
__global__ void k_check_increasing(const int32_t *X, int64_t n, int *flag) {
  GRID_STRIDE(i, n - 1) if (X[i] >= X[i + 1]) atomicOr(flag, 4);
}

void launch_gather_len(const int64_t *Ap, const int32_t *I, int64_t nI, int64_t *G, cudaStream_t st) {
  if (nI <= 0) return;
  count_launch();
  k_gather_len<<<grid1(nI), 256, 0, st>>>(Ap, I, nI, G);
}
void launch_row_starts(const int64_t *G, int64_t nI, int64_t total, int64_t *inc, cudaStream_t st) {
  if (nI <= 0 || total <= 0) return;
  count_launch();
  k_row_starts<<<grid1(nI), 256, 0, st>>>(G, nI, total, inc);
}
void launch_gather_w(const GatherArgs &a, int64_t *W, cudaStream_t st) {
  if (a.total <= 0) return;
  count_launch();
  k_gather_w<<<grid1(a.total), 256, 0, st>>>(a, W);
}
void launch_gather_fill(const GatherArgs &a, const int64_t *W, int32_t *ti, int32_t *pj, void *tv, cudaStream_t st) {
  if (a.total <= 0) return;
  count_launch();
  k_gather_fill<<<grid1(a.total), 256, 0, st>>>(a, W, ti, pj, tv);
}
void launch_gather_direct(const GatherArgs &a, const int64_t *W, int32_t *Bj, void *Bv, cudaStream_t st) {
  if (a.total <= 0) return;
  count_launch();
  k_gather_direct<<<grid1(a.total), 256, 0, st>>>(a, W, Bj, Bv);
}
void launch_gather_offsets(const int64_t *G, int64_t nI, const int64_t *W, int64_t *Bp, cudaStream_t st) {
  count_launch();
  k_gather_offsets<<<grid1(nI + 1), 256, 0, st>>>(G, nI, W, Bp);
}
void launch_check_increasing(const int32_t *X, int64_t n, int *flag, cudaStream_t st) {
  if (n <= 1) return;
  count_launch();
  k_check_increasing<<<grid1(n - 1), 256, 0, st>>>(X, n, flag);
}

// flag bit 1: an index outside [0, bound)
__global__ void k_check_range(const int32_t *X, int64_t n, int64_t bound, int *flag) {
  GRID_STRIDE(i, n) {
    const int32_t v = X[i];
    if (v < 0 || v >= bound) atomicOr(flag, 1);
  }
}
void launch_check_range(const int32_t *X, int64_t n, int64_t bound, int *flag, cudaStream_t st) {
  if (n > 0) {
    count_launch();
    k_check_range<<<grid1(n), 256, 0, st>>>(X, n, bound, flag);
  }
}

// pos[X[i]] = i (pos pre-filled with -1) for indices inside [0, bound);
// flag bit 1: an index out of range (skipped), bit 2: a repeated index.
__global__ void k_mark_positions(const int32_t *X, int64_t n, int64_t bound, int32_t *pos, int *flag) {
  GRID_STRIDE(i, n) {
    const int32_t v = X[i];
    if (v < 0 || v >= bound) {
      atomicOr(flag, 1);
      continue;
    }
    const int32_t old = atomicExch(pos + v, (int32_t)i);
    if (old != -1) atomicOr(flag, 2);
  }
}
void launch_mark_positions(const int32_t *X, int64_t n, int64_t bound, int32_t *pos, int *flag, cudaStream_t st) {
  if (n > 0) {
    count_launch();
    k_mark_positions<<<grid1(n), 256, 0, st>>>(X, n, bound, pos, flag);
  }
}

// SpAsgn R = sparse(I, 1:mb, 1, ma, mb) from rpos: counts, then entries
__global__ void k_rows_from_pos(const int32_t *pos, int64_t m, int64_t *cnt) {
  GRID_STRIDE(r, m) cnt[r + 1] = pos[r] >= 0 ? 1 : 0;
}
__global__ void k_fill_from_pos(const int32_t *pos, int64_t m, const int64_t *ptr, int32_t *out) {
  GRID_STRIDE(r, m) if (pos[r] >= 0) out[ptr[r]] = pos[r];
}
void launch_rows_from_pos(const int32_t *pos, int64_t m, int64_t *cnt, cudaStream_t st) {
  if (m > 0) {
    count_launch();
    k_rows_from_pos<<<grid1(m), 256, 0, st>>>(pos, m, cnt);
  }
}
void launch_fill_from_pos(const int32_t *pos, int64_t m, const int64_t *ptr, int32_t *out, cudaStream_t st) {
  if (m > 0) {
    count_launch();
    k_fill_from_pos<<<grid1(m), 256, 0, st>>>(pos, m, ptr, out);
  }
}
__global__ void k_add_i64(int64_t *p, int64_t n, int64_t add) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] += add;
}

void launch_add_i64(int64_t *p, int64_t n, int64_t add, cudaStream_t st) {
  if (n <= 0) return;
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (g > cap) g = cap;
  count_launch();
  k_add_i64<<<(int)g, 256, 0, st>>>(p, n, add);
}

void launch_iota_i64(int64_t *p, int64_t n, cudaStream_t st) {
  if (n > 0) {
    count_launch();
    k_iota_i64<<<grid1(n), 256, 0, st>>>(p, n);
  }
}

// ------------------------------------------------------------ SpAsgn merge

// extend-add collision: x (from A) (+) y (from B) in the semiring's add
__device__ void combine_val(const AsgnArgs &a, int64_t di, int64_t ai, int64_t xi) {
  const bool mn = a.add_kind == MIN_PLUS;
  switch (a.dtype) {
    case 0: {
      const double x = ((const double *)a.Av)[ai], y = ((const double *)a.Xv)[xi];
      ((double *)a.Cv)[di] = mn ? (y < x ? y : x) : x + y;
      break;
    }
    case 1: {
      const float x = ((const float *)a.Av)[ai], y = ((const float *)a.Xv)[xi];
      ((float *)a.Cv)[di] = mn ? (y < x ? y : x) : __fadd_rn(x, y);
      break;
    }
    case 2: {
      const int32_t x = ((const int32_t *)a.Av)[ai], y = ((const int32_t *)a.Xv)[xi];
      ((int32_t *)a.Cv)[di] = mn ? (y < x ? y : x) : (int32_t)((uint32_t)x + (uint32_t)y);
      break;
    }
    case 3: {
      const int64_t x = ((const int64_t *)a.Av)[ai], y = ((const int64_t *)a.Xv)[xi];
      ((int64_t *)a.Cv)[di] = mn ? (y < x ? y : x) : (int64_t)((unsigned long long)x + (unsigned long long)y);
      break;
    }
    default: break;
  }
}

// count: output entries of row r go to Cp[r+1]
__global__ void k_asgn_count(AsgnArgs a) {
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < a.m; r += (int64_t)gridDim.x * wpb) {
    const int64_t a0 = a.Ap[r], a1 = a.Ap[r + 1];
    const int64_t x0 = a.Xp[r], x1 = a.Xp[r + 1];
    int64_t cnt;
    if (a.rpos[r] < 0) {
      cnt = a1 - a0;  // r is not in I: R*B*Q's row is empty
    } else if (!a.accumulate) {
      long long kept = 0;
      for (int64_t q = a0 + lane; q < a1; q += 32) kept += a.cpos[a.Aj[q]] < 0;
      kept = warp_sum(kept);
      cnt = kept + (x1 - x0);
    } else {
      long long both = 0;  // columns present in A(r,:) and in R*B*Q(r,:)
      for (int64_t x = x0 + lane; x < x1; x += 32) {
        const int c = a.Xj[x];
        const int64_t at = lower_bound_col(a.Aj, a0, a1, c);
        both += (at < a1 && a.Aj[at] == c);
      }
      both = warp_sum(both);
      cnt = (a1 - a0) + (x1 - x0) - both;
    }
    if (lane == 0) a.Cp[r + 1] = cnt;
  }
}

__global__ void k_asgn_fill(AsgnArgs a) {
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < a.m; r += (int64_t)gridDim.x * wpb) {
    const int64_t a0 = a.Ap[r], a1 = a.Ap[r + 1];
    const int64_t x0 = a.Xp[r], x1 = a.Xp[r + 1];
    const int64_t o = a.Cp[r];
    if (a.rpos[r] < 0) {  // copy the row
      for (int64_t q = lane; q < a1 - a0; q += 32) {
        a.Cj[o + q] = a.Aj[a0 + q];
        copy_val(a.Cv, o + q, a.Av, a0 + q, a.vbytes);
      }
      continue;
    }
    if (lane != 0) continue;
    // merge A(r,:) (minus the I x J block when assigning) with R*B*Q(r,:)
    int64_t i = a0, x = x0, w = o;
    while (true) {
      if (!a.accumulate)
        while (i < a1 && a.cpos[a.Aj[i]] >= 0) ++i;
      const bool ha = i < a1, hx = x < x1;
      if (!ha && !hx) break;
      const int ca = ha ? a.Aj[i] : 0x7fffffff, cx = hx ? a.Xj[x] : 0x7fffffff;
      if (ca < cx) {
        a.Cj[w] = ca;
        copy_val(a.Cv, w, a.Av, i, a.vbytes);
        ++i;
      } else if (cx < ca) {
        a.Cj[w] = cx;
        copy_val(a.Cv, w, a.Xv, x, a.vbytes);
        ++x;
      } else {  // only with accumulate
        a.Cj[w] = ca;
        combine_val(a, w, i, x);
        ++i;
        ++x;
      }
      ++w;
    }
  }
}

void launch_asgn_count(const AsgnArgs &a, cudaStream_t st) {
  if (a.m > 0) {
    count_launch();
    k_asgn_count<<<grid1(a.m * 32), 256, 0, st>>>(a);
  }
}
void launch_asgn_fill(const AsgnArgs &a, cudaStream_t st) {
  if (a.m > 0) {
    count_launch();
    k_asgn_fill<<<grid1(a.m * 32), 256, 0, st>>>(a);
  }
}

}  // namespace hs
