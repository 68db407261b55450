// noalloc.cu -- hs_spgemm_noalloc: the SpGEMM pipeline with no allocation.
//
// Some callers cannot allocate device memory while they run: code that has
// handed all of the GPU's memory to its own pool and must not fragment it,
// code running inside an allocator's callback, or code that must keep its
// memory footprint fixed.  This entry point serves them.  The caller passes
// the inputs and ready-made output arrays (with their capacity); every
// temporary the product needs (flop counts, bin lists, histogram slots,
// column-segment counts, scan partials, counters) is carved from one
// file-scope device array of fixed size, and host-side readbacks go to
// ordinary (pageable) host memory.  No cudaMalloc, cudaFree, pinned-host
// allocation or allocator callback is used.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears what must start at zero.  Calls that overlap on
// the GPU (two streams, or two host threads, on one device) race on it and
// must be serialised by the caller.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/hspgemm.h"
#include "internal.h"

namespace hs {

// the fixed scratch: every GPU that loads the library holds it until exit
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)HS_NOALLOC_SCRATCH_MAX;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: its device address is looked up once per device (with that device
// current) and cached here.
constexpr int MAX_DEVICES = 64;
static std::mutex g_na_mu;
static void *g_na_ptr[MAX_DEVICES];
static bool g_na_ready[MAX_DEVICES];

static int noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HS_ECUDA;
  std::lock_guard<std::mutex> g(g_na_mu);
  if (!g_na_ready[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HS_ECUDA;
    }
    g_na_ptr[dev] = p;
    g_na_ready[dev] = true;
  }
  *out = g_na_ptr[dev];
  return HS_OK;
}

// bump allocation inside the fixed scratch
struct Arena {
  unsigned char *base;
  size_t cap, off = 0;
  bool over = false;
  size_t need = 0;
  template <typename T> T *take(size_t count) {
    const size_t bytes = ((sizeof(T) * (count ? count : 1)) + 255) & ~(size_t)255;
    need = off + bytes;
    if (off + bytes > cap) {
      over = true;
      return nullptr;
    }
    T *p = reinterpret_cast<T *>(base + off);
    off += bytes;
    return p;
  }
};

struct NaBlock {  // device counters, read back to host memory
  int key_cnt[NKEYS];
  int key_off[NKEYS + 1];
  int key_cur[NKEYS];
  int dyn[2];
  int nhist;
  int err;
  int pad[2];
  unsigned long long stats[4];
  long long nnz;
  long long dbg[2];
};

static int cuda_fail(cudaError_t e) {
  (void)e;
  cudaGetLastError();
  return HS_ECUDA;
}
#define NA_CK(call)                              \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

static int na_vbytes(int dt) {
  switch (dt) {
    case HS_F64: case HS_I64: return 8;
    case HS_F32: case HS_I32: return 4;
    default: return 0;
  }
}

static bool na_supported(int sr, int adt, int bdt, int &out_dt) {
  switch (sr) {
    case HS_PLUS_TIMES: out_dt = adt; return adt == bdt && (adt == HS_F64 || adt == HS_F32 || adt == HS_I64);
    case HS_MIN_PLUS: out_dt = adt; return adt == bdt && (adt == HS_F32 || adt == HS_I32);
    case HS_OR_AND: out_dt = HS_BOOL; return true;
    case HS_SELECT2ND: out_dt = bdt; return true;
    case HS_SELECT1ST: out_dt = adt; return true;
  }
  return false;
}

static bool na_launch_num(int sr, int out_dt, int kind, const NumArgs &a, cudaStream_t st) {
  switch (sr) {
    case HS_PLUS_TIMES: return launch_numeric_pt(out_dt, kind, a, st);
    case HS_MIN_PLUS: return launch_numeric_mp(out_dt, kind, a, st);
    case HS_OR_AND: return launch_numeric_oa(kind, a, st);
    case HS_SELECT2ND: return launch_numeric_sel(1, na_vbytes(out_dt), kind, a, st);
    case HS_SELECT1ST: return launch_numeric_sel(0, na_vbytes(out_dt), kind, a, st);
  }
  return false;
}

static int check_last() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && attr_error() != cudaSuccess) {
    e = attr_error();
    attr_error() = cudaSuccess;
  }
  return e == cudaSuccess ? HS_OK : HS_ECUDA;
}

static int spgemm_noalloc_impl(int sr, const hs_mat *A, const hs_mat *B, hs_mat *C, int64_t capacity,
                               cudaStream_t st) {
  if (!A || !B || !C) return HS_EINVAL;
  if (A->fmt != HS_CSR && A->fmt != HS_DCSR) return HS_EINVAL;
  if (B->fmt != HS_CSR) return HS_EINVAL;
  if (A->dtype < HS_F64 || A->dtype > HS_BOOL || B->dtype < HS_F64 || B->dtype > HS_BOOL) return HS_EINVAL;
  if (A->n != B->m || A->m < 0 || B->n < 0 || A->nnz < 0 || B->nnz < 0 || capacity < 0) return HS_EINVAL;
  if (B->n > 0x7fffffffLL || A->n > 0x7fffffffLL) return HS_EINVAL;
  int out_dt = 0;
  if (!na_supported(sr, A->dtype, B->dtype, out_dt)) return HS_EINVAL;
  const int vb = na_vbytes(out_dt);
  if ((sr == HS_PLUS_TIMES || sr == HS_MIN_PLUS) && ((A->nnz && !A->val) || (B->nnz && !B->val))) return HS_EINVAL;
  if (sr == HS_SELECT2ND && vb && B->nnz && !B->val) return HS_EINVAL;
  if (sr == HS_SELECT1ST && vb && A->nnz && !A->val) return HS_EINVAL;
  const int64_t m = A->m, n = B->n;
  const int64_t nslots = A->fmt == HS_DCSR ? A->nzr : A->m;
  if (nslots < 0 || (A->fmt == HS_DCSR && nslots > 0 && !A->ids)) return HS_EINVAL;
  if (nslots > 0x7fffffffLL) return HS_EUNSUPPORTED;
  // every input array a kernel will read must be there: checked before the first CUDA call
  if ((nslots > 0 && !A->ptr) || (B->m > 0 && !B->ptr)) return HS_EINVAL;
  if ((A->nnz > 0 && !A->idx) || (B->nnz > 0 && !B->idx)) return HS_EINVAL;
  if (!C->ptr || (capacity > 0 && (!C->idx || (vb && !C->val)))) return HS_EINVAL;

  C->fmt = HS_CSR;
  C->dtype = out_dt;
  C->m = m;
  C->n = n;
  C->nnz = 0;
  C->nzr = 0;
  C->ids = nullptr;
  if (!vb) C->val = nullptr;
  int64_t *Cp = C->ptr;
  NA_CK(cudaMemsetAsync(Cp, 0, sizeof(int64_t) * (size_t)(m + 1), st));
  if (nslots == 0 || A->nnz == 0 || B->nnz == 0 || n == 0) return check_last();

  void *sp = nullptr;
  if (int e = noalloc_scratch(&sp)) return e;
  Arena ar{reinterpret_cast<unsigned char *>(sp), NOALLOC_SCRATCH_BYTES};
  NaBlock *sb = ar.take<NaBlock>(1);
  int64_t *f = ar.take<int64_t>(nslots);
  int *list = ar.take<int>(nslots);
  int32_t *hslot = ar.take<int32_t>(nslots);
  int64_t *scan_tmp = ar.take<int64_t>(scan_tmp_elems(m + 1));
  if (ar.over) return HS_ESCRATCH;
  static thread_local NaBlock hb;  // host copy (ordinary memory)

  const BinCfg bins = product_bins(bin_config(vb), n, vb);
  RowSet rs{A->ptr, A->idx, A->val, A->fmt == HS_DCSR ? A->ids : nullptr, nslots, A->nnz, m, sb->dbg};
  RightOp rb{B->ptr, B->idx, B->val, n, B->m, B->nnz, sb->dbg};
  NA_CK(cudaMemsetAsync(sb, 0, sizeof(NaBlock), st));
  launch_flops(rs, rb, f, sb->key_cnt, sb->stats, bins, st);
  launch_key_offsets(sb->key_cnt, sb->key_off, sb->key_cur, st);
  launch_scatter_sym(rs, f, sb->key_cur, list, hslot, &sb->nhist, bins, st);
  if (int e = check_last()) return e;
  NA_CK(cudaMemcpyAsync(&hb, sb, sizeof(NaBlock), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (hb.stats[1] >= (1ull << 31)) return HS_EUNSUPPORTED;
  int key_off[NKEYS + 1];
  memcpy(key_off, hb.key_off, sizeof(key_off));
  const int nhist = hb.nhist;
  const int nseg = (int)((n + SEG_W - 1) / SEG_W);
  uint32_t *hist = nullptr;
  if (nhist > 0) {
    hist = ar.take<uint32_t>((size_t)nhist * nseg);
    if (ar.over) return HS_ESCRATCH;
    NA_CK(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)nhist * nseg, st));
  }

  SymArgs sa{rs, rb, f, nullptr, 0, Cp, hslot, hist, nseg, &sb->dyn[0], &sb->err, nullptr, nullptr, nullptr, 0};
  auto sym_bin = [&](int k0, int k1) {
    sa.list = list + key_off[k0];
    sa.count = key_off[k1] - key_off[k0];
  };
  sym_bin(KEY_TINY, KEY_TINY + 1);
  launch_sym_tiny(sa, st);
  sym_bin(KEY_WARP, KEY_WARP + 1);
  launch_sym_warp(sa, st);
  sym_bin(KEY_MID_S, KEY_MID_S + 1);
  launch_sym_mid_s(sa, st);
  sym_bin(KEY_MID, KEY_MID + 1);
  launch_sym_mid(sa, st);
  sym_bin(KEY_LARGE, KEY_LARGE + 1);
  launch_sym_large(sa, st);
  sym_bin(KEY_SPA, KEY_SPA + 1);
  launch_sym_spa(sa, st);
  sym_bin(KEY_HEAVY, NKEYS);
  launch_sym_heavy(sa, st);
  if (int e = check_last()) return e;

  launch_scan_i64(Cp, m + 1, scan_tmp, st);
  NA_CK(cudaMemsetAsync(sb->key_cnt, 0, sizeof(int) * NKEYS, st));
  launch_num_count(rs, f, Cp, numeric_bins(bins, n), sb->key_cnt, st);
  launch_key_offsets(sb->key_cnt, sb->key_off, sb->key_cur, st);
  launch_scatter_num(rs, f, Cp, numeric_bins(bins, n), sb->key_cur, list, st);
  NA_CK(cudaMemcpyAsync(&sb->nnz, Cp + m, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  if (int e = check_last()) return e;
  NA_CK(cudaMemcpyAsync(&hb, sb, sizeof(NaBlock), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (hb.dbg[0] || hb.err) return HS_EINTERNAL;
  C->nnz = hb.nnz;
  if (hb.nnz > capacity) return HS_ECAPACITY;  // C->ptr is complete, C->nnz is the size needed
  memcpy(key_off, hb.key_off, sizeof(key_off));

  int32_t *gcur = nullptr, *gend = nullptr;
  if (key_off[NKEYS] > key_off[KEY_HEAVY]) {
    gcur = ar.take<int32_t>((size_t)A->nnz);
    gend = ar.take<int32_t>((size_t)A->nnz);
    if (ar.over) {
      C->nnz = 0;  // C->ptr holds the row offsets, but no entry was written
      return HS_ESCRATCH;
    }
  }
  NumArgs na{rs,   rb,   f,    nullptr,     0,        Cp,   C->idx, C->val,  hslot,
             hist, nseg, &sb->dyn[1], &sb->err, gcur, gend, nullptr, nullptr, nullptr, nullptr};
  for (int kind = 0; kind < NUM_KINDS; ++kind) {
    const int k0 = KEY_TINY + kind, k1 = kind == NUM_KINDS - 1 ? NKEYS : k0 + 1;
    na.list = list + key_off[k0];
    na.count = key_off[k1] - key_off[k0];
    if (na.count > 0 && !na_launch_num(sr, out_dt, kind, na, st)) return HS_EINVAL;
  }
  if (int e = check_last()) return e;
  NA_CK(cudaMemcpyAsync(&hb, sb, sizeof(NaBlock), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (hb.dbg[0] || hb.err) return HS_EINTERNAL;
  return HS_OK;
}

}  // namespace hs

extern "C" int hs_spgemm_noalloc(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C, int64_t capacity,
                                 void *stream) {
  return hs::spgemm_noalloc_impl(semiring, A, B, C, capacity, (cudaStream_t)stream);
}
