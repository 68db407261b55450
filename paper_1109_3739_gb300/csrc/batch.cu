// batch.cu -- hs_spgemm_batched: many independent products C_i = A_i * B_i.
//
// The problems are run as one block-diagonal product: the A_i are stacked
// into one row set whose column ids are shifted to the stacked rows of the
// B_i, and one pass of the binned SpGEMM pipeline (flops, bins, symbolic,
// scan, numeric) serves every row of every problem.  Rows of all problems mix
// in the same bins, so small and large problems share launches and the GPU
// stays full however uneven the sizes are; the whole batch costs one launch
// per phase and two host synchronisations instead of that many per problem.
// The output is the stacked C (local column ids): C_i is rows
// row_offsets[i] .. row_offsets[i+1] of it.
#include <cstring>
#include <vector>

#include "../../include/hspgemm.h"
#include "internal.h"

namespace hs {

struct BatchDesc {
  const int64_t *ap, *bp;  // row offsets of A_i, B_i
  const int32_t *aj, *bj;  // column ids
  const void *av, *bv;     // values (may be null)
  int64_t a_row0, a_nnz0;  // where A_i starts in the stacked A (rows, entries)
  int64_t b_row0, b_nnz0;  // where B_i starts in the stacked B
  int64_t am, bm;          // rows of A_i, B_i
};

// index of the problem whose range [off[p], off[p+1]) holds x
__device__ __forceinline__ int find_problem(const int64_t *off, int count, int64_t x) {
  int lo = 0, hi = count;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

#define GRID_STRIDE64(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// stacked row offsets: which = 0 for A, 1 for B
__global__ void k_batch_rows(const BatchDesc *d, const int64_t *row_off, int count, int which, int64_t rows,
                             int64_t total_nnz, int64_t *ptr) {
  GRID_STRIDE64(r, rows + 1) {
    if (r == rows) {
      ptr[r] = total_nnz;
      continue;
    }
    const int p = find_problem(row_off, count, r);
    const BatchDesc &b = d[p];
    const int64_t local = r - (which ? b.b_row0 : b.a_row0);
    ptr[r] = (which ? b.bp[local] - b.bp[0] + b.b_nnz0 : b.ap[local] - b.ap[0] + b.a_nnz0);
  }
}

// stacked entries; A's column ids move to the stacked rows of B
__global__ void k_batch_entries(const BatchDesc *d, const int64_t *nnz_off, int count, int which, int64_t nnz,
                                int vbytes, int32_t *j, void *v) {
  GRID_STRIDE64(q, nnz) {
    const int p = find_problem(nnz_off, count, q);
    const BatchDesc &b = d[p];
    if (which == 0) {
      const int64_t src = b.ap[0] + (q - b.a_nnz0);
      j[q] = b.aj[src] + (int32_t)b.b_row0;
      if (vbytes == 8) reinterpret_cast<unsigned long long *>(v)[q] = reinterpret_cast<const unsigned long long *>(b.av)[src];
      else if (vbytes == 4) reinterpret_cast<uint32_t *>(v)[q] = reinterpret_cast<const uint32_t *>(b.av)[src];
    } else {
      const int64_t src = b.bp[0] + (q - b.b_nnz0);
      j[q] = b.bj[src];
      if (vbytes == 8) reinterpret_cast<unsigned long long *>(v)[q] = reinterpret_cast<const unsigned long long *>(b.bv)[src];
      else if (vbytes == 4) reinterpret_cast<uint32_t *>(v)[q] = reinterpret_cast<const uint32_t *>(b.bv)[src];
    }
  }
}

static int bgrid(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

static int vb_of(int dt) {
  switch (dt) {
    case HS_F64: case HS_I64: return 8;
    case HS_F32: case HS_I32: return 4;
    default: return 0;
  }
}

}  // namespace hs

using namespace hs;

extern "C" int hs_batch_stack(int64_t count, const hs_mat *A, const hs_mat *B, hs_mat *SA, hs_mat *SB,
                              int64_t *row_offsets, const hs_allocator *al, void *stream) {
  if (!SA || !SB || count < 0 || (count > 0 && (!A || !B || !row_offsets))) return HS_EINVAL;
  if (count > 0x7fffffffLL) return HS_EUNSUPPORTED;
  memset(SA, 0, sizeof(*SA));
  memset(SB, 0, sizeof(*SB));
  cudaStream_t st = (cudaStream_t)stream;
  // host-side layout of the stacked operands
  std::vector<BatchDesc> d((size_t)count);
  std::vector<int64_t> a_row(count + 1, 0), a_nnz(count + 1, 0), b_row(count + 1, 0), b_nnz(count + 1, 0);
  int64_t nmax = 0;
  for (int64_t i = 0; i < count; ++i) {
    const hs_mat &a = A[i], &b = B[i];
    if (a.fmt != HS_CSR || b.fmt != HS_CSR || a.n != b.m || a.m < 0 || b.n < 0) return HS_EINVAL;
    if (a.dtype != A[0].dtype || b.dtype != B[0].dtype) return HS_EINVAL;
    if ((a.m > 0 && !a.ptr) || (b.m > 0 && !b.ptr)) return HS_EINVAL;
    if ((a.nnz > 0 && !a.idx) || (b.nnz > 0 && !b.idx)) return HS_EINVAL;
    a_row[i + 1] = a_row[i] + a.m;
    a_nnz[i + 1] = a_nnz[i] + a.nnz;
    b_row[i + 1] = b_row[i] + b.m;
    b_nnz[i + 1] = b_nnz[i] + b.nnz;
    if (b.n > nmax) nmax = b.n;
    d[i] = BatchDesc{a.ptr, b.ptr, a.idx, b.idx, a.val, b.val, a_row[i], a_nnz[i], b_row[i], b_nnz[i], a.m, b.m};
  }
  if (b_row[count] > 0x7fffffffLL) return HS_EUNSUPPORTED;  // stacked column ids of A are int32
  const int adt = count ? A[0].dtype : HS_F64, bdt = count ? B[0].dtype : HS_F64;
  const int avb = (adt == HS_BOOL) ? 0 : vb_of(adt), bvb = (bdt == HS_BOOL) ? 0 : vb_of(bdt);
  for (int64_t i = 0; i < count; ++i) {
    if (avb && A[i].nnz && !A[i].val) return HS_EINVAL;
    if (bvb && B[i].nnz && !B[i].val) return HS_EINVAL;
  }
  for (int64_t i = 0; i <= count; ++i) row_offsets[i] = a_row[i];

  // outputs and temporaries through the caller's allocator (or cudaMallocAsync)
  auto alloc = [&](size_t bytes) -> void * {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (al && al->alloc) p = al->alloc(bytes, stream, al->ctx);
    else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p;
  };
  auto release = [&](void *p, size_t bytes) {
    if (!p) return;
    if (al && al->free) al->free(p, bytes ? bytes : 16, stream, al->ctx);
    else if (!al || !al->alloc) cudaFreeAsync(p, st);
  };
  struct Blk {
    void *p;
    size_t n;
  };
  std::vector<Blk> temps, outs;
  auto take = [&](std::vector<Blk> &v, size_t bytes) -> void * {
    void *p = alloc(bytes);
    if (p) v.push_back({p, bytes ? bytes : 16});
    return p;
  };
  const int64_t am = a_row[count], annz = a_nnz[count], bm = b_row[count], bnnz = b_nnz[count];
  int status = HS_OK;
  do {
    BatchDesc *dd = (BatchDesc *)take(temps, sizeof(BatchDesc) * (size_t)(count ? count : 1));
    int64_t *offs = (int64_t *)take(temps, sizeof(int64_t) * 4 * (size_t)(count + 1));
    int64_t *Ap = (int64_t *)take(outs, sizeof(int64_t) * (size_t)(am + 1));
    int32_t *Aj = (int32_t *)take(outs, sizeof(int32_t) * (size_t)annz);
    void *Av = avb ? take(outs, (size_t)avb * (size_t)annz) : nullptr;
    int64_t *Bp = (int64_t *)take(outs, sizeof(int64_t) * (size_t)(bm + 1));
    int32_t *Bj = (int32_t *)take(outs, sizeof(int32_t) * (size_t)bnnz);
    void *Bv = bvb ? take(outs, (size_t)bvb * (size_t)bnnz) : nullptr;
    if (!dd || !offs || !Ap || !Aj || !Bp || !Bj || (avb && !Av) || (bvb && !Bv)) {
      status = HS_ENOMEM;
      break;
    }
    if (count > 0) {
      std::vector<int64_t> h(4 * (size_t)(count + 1));
      memcpy(h.data(), a_row.data(), 8 * (count + 1));
      memcpy(h.data() + (count + 1), a_nnz.data(), 8 * (count + 1));
      memcpy(h.data() + 2 * (count + 1), b_row.data(), 8 * (count + 1));
      memcpy(h.data() + 3 * (count + 1), b_nnz.data(), 8 * (count + 1));
      if (cudaMemcpyAsync(dd, d.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(offs, h.data(), 8 * h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        status = HS_ECUDA;
        break;
      }
      const int cnt = (int)count;
      count_launch();
      k_batch_rows<<<bgrid(am + 1), 256, 0, st>>>(dd, offs, cnt, 0, am, annz, Ap);
      count_launch();
      k_batch_rows<<<bgrid(bm + 1), 256, 0, st>>>(dd, offs + 2 * (count + 1), cnt, 1, bm, bnnz, Bp);
      if (annz > 0) {
        count_launch();
        k_batch_entries<<<bgrid(annz), 256, 0, st>>>(dd, offs + (count + 1), cnt, 0, annz, avb, Aj, Av);
      }
      if (bnnz > 0) {
        count_launch();
        k_batch_entries<<<bgrid(bnnz), 256, 0, st>>>(dd, offs + 3 * (count + 1), cnt, 1, bnnz, bvb, Bj, Bv);
      }
      // (copies from pageable host memory return once the source is staged,
      // so the host vectors may go out of scope)
      if (cudaGetLastError() != cudaSuccess) {
        status = HS_ECUDA;
        break;
      }
    } else {
      cudaMemsetAsync(Ap, 0, 8, st);
      cudaMemsetAsync(Bp, 0, 8, st);
    }
    *SA = hs_mat{HS_CSR, adt, am, bm, annz, 0, Ap, Aj, nullptr, Av};
    *SB = hs_mat{HS_CSR, bdt, bm, nmax, bnnz, 0, Bp, Bj, nullptr, Bv};
  } while (0);
  for (auto &b : temps) release(b.p, b.n);
  if (status != HS_OK) {
    for (auto &b : outs) release(b.p, b.n);
    memset(SA, 0, sizeof(*SA));
    memset(SB, 0, sizeof(*SB));
  }
  return status;
}

extern "C" int hs_spgemm_batched(int semiring, int64_t count, const hs_mat *A, const hs_mat *B, hs_mat *C,
                                 int64_t *row_offsets, const hs_allocator *al, void *stream, uint32_t flags) {
  if (!C) return HS_EINVAL;
  memset(C, 0, sizeof(*C));
  hs_mat SA, SB;
  int status = hs_batch_stack(count, A, B, &SA, &SB, row_offsets, al, stream);
  if (status != HS_OK) return status;
  status = hs_spgemm(semiring, &SA, &SB, C, al, stream, flags);
  hs_mat_free(&SA, al, stream);
  hs_mat_free(&SB, al, stream);
  return status;
}
