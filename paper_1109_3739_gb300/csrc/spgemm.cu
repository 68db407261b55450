// spgemm.cu -- host driver and C ABI (include/hspgemm.h).
//
// hs_spgemm runs the phases of the row-wise SpGEMM on one stream:
//   1. flops per row and binning of the non-empty rows by flops
//      (one device->host read: bin sizes, total flops, validation flags);
//   2. symbolic pass per bin: output nonzeros per row;
//   3. inclusive scan of the counts into C's row offsets, binning of the rows
//      again by (flops, output count) for the numeric pass
//      (second device->host read: nnz(C) and the bin sizes);
//   4. allocation of C's column ids and values, numeric pass per bin.
// hs_spref and hs_spasgn build their 0/1 selection matrices on the device and
// call the same driver with the selector semirings (Section 3.1).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/hspgemm.h"
#include "internal.h"

namespace hs {

static thread_local int t_last_cuda = 0;
static thread_local char t_detail[256] = "";

// Checking mode: HS_DEBUG_SYNC=1 in the environment synchronises after every
// phase, so a CUDA error or a failed index check is attributed to the phase
// that raised it.  Without it, failed checks are reported at the product's
// second host synchronisation (or at the end with HS_FLAG_VALIDATE).
static bool debug_sync() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("HS_DEBUG_SYNC");
    v = (e && *e && *e != '0') ? 1 : 0;
  }
  return v == 1;
}

// ---------------------------------------------------------------- profiling
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int64_t> launches;
  struct Pending {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  int phase_id(const char *nm) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == nm) return (int)i;
    names.push_back(nm);
    ms.push_back(0);
    launches.push_back(0);
    return (int)names.size() - 1;
  }
  void drain() {
    for (auto &p : pending) {
      cudaEventSynchronize(p.b);
      float t = 0;
      cudaEventElapsedTime(&t, p.a, p.b);
      ms[p.phase] += t;
      launches[p.phase] += 1;
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    pending.clear();
  }
};
static Prof g_prof;

struct PhaseTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  int phase = -1;
  cudaStream_t st;
  PhaseTimer(const char *nm, cudaStream_t s, bool active = true) : st(s) {
    if (!g_prof.on || !active) return;
    std::lock_guard<std::mutex> g(g_prof.mu);
    phase = g_prof.phase_id(nm);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  ~PhaseTimer() {
    if (phase < 0) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.pending.push_back({phase, a, b});
  }
};

// --------------------------------------------------------------- allocation
struct Mem {
  const hs_allocator *al;
  cudaStream_t st;
  cudaMemPool_t pool = nullptr;  // without an allocator: this pool if set, else the device's default pool
  struct Blk {
    void *p;
    size_t n;
  };
  std::vector<Blk> scratch;
  bool failed = false;

  void *raw(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (al && al->alloc) {
      p = al->alloc(bytes, (void *)st, al->ctx);
    } else if ((pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st)) !=
               cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (!p) failed = true;
    return p;
  }
  void release(void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (al && al->free) al->free(p, bytes, (void *)st, al->ctx);
    else if (!al || !al->alloc) cudaFreeAsync(p, st);
  }
  template <typename T> T *tmp(size_t count) {
    T *p = (T *)raw(sizeof(T) * count);
    if (p) scratch.push_back({p, sizeof(T) * count});
    return p;
  }
  ~Mem() {
    for (auto &b : scratch) release(b.p, b.n);
  }
};

// A pool of the library's own for calls that allocate and free the same large
// blocks many times (hs_spgemm_to_host): it keeps freed memory mapped for the
// next block and the next call (hs_trim_memory returns it) instead of giving
// it back at every synchronisation.
static cudaMemPool_t own_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
      cudaGetLastError();
      pools[dev] = nullptr;
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
  }
  return pools[dev];
}

static int vbytes_of(int dt) {
  switch (dt) {
    case HS_F64: case HS_I64: return 8;
    case HS_F32: case HS_I32: return 4;
    default: return 0;
  }
}

// pinned staging for the small device->host reads: one 8 KB page-locked
// buffer per thread, shared by every call on that thread.  A caller reads
// what it copied there before it calls another operation's implementation
// (SpAsgn runs two products, SpRef may build Q with sparse()), and copies
// into it again afterwards.
struct Pinned {
  void *p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
static thread_local Pinned t_pin;
static void *pinned(size_t bytes) {
  if (!t_pin.p && cudaMallocHost(&t_pin.p, 8192) != cudaSuccess) {
    t_pin.p = nullptr;
    return nullptr;
  }
  return bytes <= 8192 ? t_pin.p : nullptr;
}

#define CK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      t_last_cuda = (int)e_;              \
      cudaGetLastError();                 \
      return HS_ECUDA;                    \
    }                                     \
  } while (0)

static int check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && attr_error() != cudaSuccess) {
    e = attr_error();
    attr_error() = cudaSuccess;
  }
  if (e != cudaSuccess) {
    t_last_cuda = (int)e;
    snprintf(t_detail, sizeof(t_detail), "%s (%d)", cudaGetErrorName(e), (int)e);
    return HS_ECUDA;
  }
  return HS_OK;
}

struct SmallBlock;
static int phase_check(const char *phase, cudaStream_t st, const long long *dbg_dev);

static bool dtype_ok(int dt) { return dt >= HS_F64 && dt <= HS_BOOL; }

static void free_mat(hs_mat *M, Mem &mem) {
  if (!M) return;
  const int64_t rows = M->m;
  mem.release(M->ptr, sizeof(int64_t) * (size_t)(rows + 1));
  mem.release(M->idx, sizeof(int32_t) * (size_t)M->nnz);
  if (M->val) mem.release(M->val, (size_t)vbytes_of(M->dtype) * (size_t)M->nnz);
  memset(M, 0, sizeof(*M));
}

// ----------------------------------------------------------------- SpGEMM
struct SmallBlock {  // device counters, read back in one copy
  int key_cnt[NKEYS];
  int key_off[NKEYS + 1];
  int key_cur[NKEYS];
  int dyn[3];  // symbolic heavy rows, numeric heavy rows, numeric heavy units
  int nhist;
  int err;
  int valflag;
  int pad;
  unsigned long long stats[4];
  unsigned long long lpool;  // heavy rows' column lists: pool entries handed out
  int bci_cnt;               // B segment index rows handed out
  int pad2;
  long long nunits;          // numeric heavy units (column parts of rows with lists)
  long long npcap;           // their room in the pair arrays
  long long nnz;
  unsigned long long zeros;  // A entries whose B row is empty
  long long dbg[2];  // guarded builds: first failed check (code, index)
};

static int phase_check(const char *phase, cudaStream_t st, const long long *dbg_dev) {
  if (int e = check_launch()) {
    char tmp[sizeof(t_detail) + 64];
    snprintf(tmp, sizeof(tmp), "%.48s: %s", phase, t_detail);
    snprintf(t_detail, sizeof(t_detail), "%.*s", (int)sizeof(t_detail) - 1, tmp);
    return e;
  }
  if (!debug_sync()) return HS_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    t_last_cuda = (int)e;
    snprintf(t_detail, sizeof(t_detail), "%s: %s (%d)", phase, cudaGetErrorName(e), (int)e);
    cudaGetLastError();
    return HS_ECUDA;
  }
  if (dbg_dev) {
    long long d[2] = {0, 0};
    cudaMemcpy(d, dbg_dev, sizeof(d), cudaMemcpyDeviceToHost);
    if (d[0]) {
      snprintf(t_detail, sizeof(t_detail), "%s: guard %lld failed at index %lld", phase, d[0], d[1]);
      return HS_EINTERNAL;
    }
  }
  return HS_OK;
}

static bool numeric_supported(int sr, int adt, int bdt, int &out_dt) {
  switch (sr) {
    case HS_PLUS_TIMES:
      out_dt = adt;
      return adt == bdt && (adt == HS_F64 || adt == HS_F32 || adt == HS_I64);
    case HS_MIN_PLUS:
      out_dt = adt;
      return adt == bdt && (adt == HS_F32 || adt == HS_I32);
    case HS_OR_AND:
      out_dt = HS_BOOL;
      return true;
    case HS_SELECT2ND:
      out_dt = bdt;
      return true;
    case HS_SELECT1ST:
      out_dt = adt;
      return true;
  }
  return false;
}



// ----------------------------------------------------------------- tuning
static std::mutex g_tune_mu;
static const hs_tuning k_tune_default = {F_WARP_S, CAP_MID_S, 4096, F_MID_S, 0, F_SORT, 50, 0, 16, 0};
static hs_tuning g_tune = k_tune_default;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

BinCfg bin_config(int value_bytes) {
  hs_tuning t;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    t = g_tune;
  }
  BinCfg b;
  b.cap_large = value_bytes == 8 ? 4096 : 8192;
  b.warp_s_max = clampi(t.warp_s_max, F_TINY, F_WARP_S);
  b.mid_s_max = clampi(t.mid_s_max, 0, CAP_MID_S);
  b.large_s_max = clampi(t.large_s_max, CAP_MID, b.cap_large / 2 > CAP_MID ? b.cap_large / 2 : CAP_MID);
  b.sym_mid_s_max = clampi(t.sym_mid_s_max, F_WARP, F_MID_S);
  // 0: automatic.  With 4-byte values and bool, rows of more than 4096
  // products take the bitmap kernel and rows of more than 2048 outputs among
  // them the units (R-MAT scale 20: 77.8 ms against 79.0 ms with both at the
  // large capacity); 8-byte values keep the large capacity
  const bool narrow = value_bytes <= 4;
  b.sym_heavy_from = t.sym_heavy_from <= 0 ? (narrow ? F_MID : b.cap_large) : clampi(t.sym_heavy_from, 2 * F_MID_S, b.cap_large);
  b.sort_max = clampi(t.sort_max, F_TINY, F_SORT);
  b.sort_pct = clampi(t.sort_pct, 0, 101);
  b.spa_max = clampi(t.spa_max, 0, SPA_COLS_4);
  b.unit_kb = t.heavy_part_kb >= 32 ? 32 : 16;
  b.num_heavy_from =
      t.num_heavy_from <= 0 ? (narrow ? CAP_MID : b.cap_large) : clampi(t.num_heavy_from, CAP_MID, b.cap_large);
  b.spa = 0;
  return b;
}

static bool launch_num(int sr, int out_dt, int kind, const NumArgs &a, cudaStream_t st) {
  switch (sr) {
    case HS_PLUS_TIMES: return launch_numeric_pt(out_dt, kind, a, st);
    case HS_MIN_PLUS: return launch_numeric_mp(out_dt, kind, a, st);
    case HS_OR_AND: return launch_numeric_oa(kind, a, st);
    case HS_SELECT2ND: return launch_numeric_sel(1, vbytes_of(out_dt), kind, a, st);
    case HS_SELECT1ST: return launch_numeric_sel(0, vbytes_of(out_dt), kind, a, st);
  }
  return false;
}

}  // namespace hs

// A product's numeric pass, kept for re-execution (hs_plan_*): the numeric
// arguments with every scratch buffer, the row bins, and the buffers' owner.
struct hs_plan {
  int sr = 0, out_dt = 0;
  int64_t a_nnz = 0, b_nnz = 0, c_nnz = 0;
  hs::NumArgs na{};
  const int *list = nullptr;
  int off[hs::NUM_KINDS] = {0}, count[hs::NUM_KINDS] = {0};
  int *dyn = nullptr, *err = nullptr;
  long long *dbg = nullptr;
  hs_allocator al{};
  bool has_al = false;
  std::vector<hs::Mem::Blk> blocks;
};

namespace hs {

// Where C's column ids and values go when the caller places them (device
// pointers to memory of at least cap entries, e.g. host memory the GPU maps).
struct OutPlace {
  int32_t *idx;
  void *val;
  int64_t cap;
};

static int spgemm_impl(int sr, const hs_mat *A, const hs_mat *B, hs_mat *C, Mem &mem, Mem &outmem,
                       uint32_t flags, hs_plan *plan = nullptr, const OutPlace *place = nullptr) {
  cudaStream_t st = mem.st;
  if (!A || !B || !C) return HS_EINVAL;
  if (A->fmt != HS_CSR && A->fmt != HS_DCSR) return HS_EINVAL;
  if (B->fmt != HS_CSR) return HS_EINVAL;
  if (!dtype_ok(A->dtype) || !dtype_ok(B->dtype)) return HS_EINVAL;
  if (A->n != B->m || A->m < 0 || B->n < 0 || A->nnz < 0 || B->nnz < 0) return HS_EINVAL;
  if (B->n > 0x7fffffffLL || A->n > 0x7fffffffLL) return HS_EINVAL;
  int out_dt = 0;
  if (!numeric_supported(sr, A->dtype, B->dtype, out_dt)) return HS_EINVAL;
  const int vb = vbytes_of(out_dt);
  if ((sr == HS_PLUS_TIMES || sr == HS_MIN_PLUS) && ((A->nnz && !A->val) || (B->nnz && !B->val))) return HS_EINVAL;
  if (sr == HS_SELECT2ND && vb && B->nnz && !B->val) return HS_EINVAL;
  if (sr == HS_SELECT1ST && vb && A->nnz && !A->val) return HS_EINVAL;
  const int64_t m = A->m, n = B->n;
  const int64_t nslots = A->fmt == HS_DCSR ? A->nzr : A->m;
  if (nslots < 0 || (A->fmt == HS_DCSR && nslots > 0 && !A->ids)) return HS_EINVAL;
  if ((nslots > 0 && !A->ptr) || (B->m >= 0 && !B->ptr && B->m > 0)) return HS_EINVAL;
  if ((A->nnz > 0 && !A->idx) || (B->nnz > 0 && !B->idx)) return HS_EINVAL;
  if (nslots > 0x7fffffffLL) return HS_EUNSUPPORTED;

  memset(C, 0, sizeof(*C));
  C->fmt = HS_CSR;
  C->dtype = out_dt;
  C->m = m;
  C->n = n;
  int64_t *Cp = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(m + 1));
  if (!Cp) return HS_ENOMEM;
  C->ptr = Cp;
  CK(cudaMemsetAsync(Cp, 0, sizeof(int64_t) * (size_t)(m + 1), st));
  if (plan) {
    plan->sr = sr;
    plan->out_dt = out_dt;
    plan->a_nnz = A->nnz;
    plan->b_nnz = B->nnz;
  }
  if (nslots == 0 || A->nnz == 0 || B->nnz == 0 || n == 0) {
    if (place) {  // nothing to write
      C->idx = place->idx;
      C->val = place->val;
      return check_launch();
    }
    C->idx = (int32_t *)outmem.raw(4);
    if (!C->idx) return HS_ENOMEM;
    if (vb) {  // typed outputs always carry a (here empty) value array
      C->val = outmem.raw((size_t)vb);
      if (!C->val) return HS_ENOMEM;
    }
    return check_launch();
  }

  const BinCfg bins = product_bins(bin_config(vb), n, vb);
  int64_t *f = mem.tmp<int64_t>(nslots);
  int *list = mem.tmp<int>(nslots);
  int32_t *hslot = mem.tmp<int32_t>(nslots);
  SmallBlock *sb = mem.tmp<SmallBlock>(1);
  if (mem.failed) return HS_ENOMEM;
  RowSet rs{A->ptr, A->idx, A->val, A->fmt == HS_DCSR ? A->ids : nullptr, nslots, A->nnz, m, sb->dbg};
  RightOp rb{B->ptr, B->idx, B->val, n, B->m, B->nnz, sb->dbg};
  SmallBlock *hb = (SmallBlock *)pinned(sizeof(SmallBlock));
  if (!hb) return HS_ECUDA;
  CK(cudaMemsetAsync(sb, 0, sizeof(SmallBlock), st));

  // product counts per A entry and their scan: every row's count without a
  // warp walking the row (optional scratch; without it, one warp per row)
  int64_t *es = (int64_t *)mem.raw(sizeof(int64_t) * (size_t)A->nnz);
  int64_t *es_tmp = es ? (int64_t *)mem.raw(sizeof(int64_t) * (size_t)scan_tmp_elems(A->nnz)) : nullptr;
  if (es) mem.scratch.push_back({es, sizeof(int64_t) * (size_t)A->nnz});
  if (es_tmp) mem.scratch.push_back({es_tmp, sizeof(int64_t) * (size_t)scan_tmp_elems(A->nnz)});
  mem.failed = false;
  const bool flat = es && es_tmp;
  {
    PhaseTimer t("analysis", st);
    if (flags & HS_FLAG_VALIDATE) {
      launch_validate(A->ptr, A->idx, nslots, A->n, &sb->valflag, st);
      launch_validate(B->ptr, B->idx, B->m, B->n, &sb->valflag, st);
    }
    if (flat) {
      launch_entry_flops(rs, rb, es, &sb->zeros, st);
      launch_scan_i64(es, A->nnz, es_tmp, st);
      launch_row_flops(rs, es, f, sb->key_cnt, sb->stats, bins, B->n, st);
    } else {
      launch_flops(rs, rb, f, sb->key_cnt, sb->stats, bins, st);
    }
    launch_key_offsets(sb->key_cnt, sb->key_off, sb->key_cur, st);
    launch_scatter_sym(rs, f, sb->key_cur, list, hslot, &sb->nhist, bins, st);
  }
  if (int e = phase_check("analysis", st, sb->dbg)) return e;
  CK(cudaMemcpyAsync(hb, sb, sizeof(SmallBlock), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hb->valflag & 4) return HS_EINVAL;
  if (hb->valflag & 1) return HS_EINVAL;
  if (hb->valflag & 2) return HS_ENONCANON;
  if (hb->stats[1] >= (1ull << 31)) return HS_EUNSUPPORTED;  // one row's products must fit int32
  int key_off[NKEYS + 1];
  memcpy(key_off, hb->key_off, sizeof(key_off));
  const int nhist = hb->nhist;
  const int nseg = (int)((n + SEG_W - 1) / SEG_W);

  // A entries whose B row is empty make no products.  When they are most of
  // a large A (a very sparse B, as in the tall-skinny products of Section 4),
  // the passes below read a copy of A without them: rows keep their product
  // counts, bins and results, and a long row of A with few products no longer
  // costs a walk over all its entries.  Not for plans, whose execute reads A's
  // values in place.
  if (flat && !plan && A->nnz >= (1 << 20) && hb->zeros * 2 > (unsigned long long)A->nnz) {
    const int64_t kept = A->nnz - (int64_t)hb->zeros;
    const int va = A->val ? vbytes_of(A->dtype) : 0;
    int64_t *keep = mem.tmp<int64_t>((size_t)A->nnz);
    int32_t *j2 = mem.tmp<int32_t>((size_t)(kept > 0 ? kept : 1));
    void *v2 = va ? (void *)mem.tmp<char>((size_t)va * (size_t)(kept > 0 ? kept : 1)) : nullptr;
    int64_t *p2 = mem.tmp<int64_t>((size_t)nslots + 1);
    if (!mem.failed) {
      PhaseTimer t("compact_a", st);
      launch_compact_a(rs, es, keep, es_tmp, j2, v2, va, p2, st);
      rs.p = p2;
      rs.j = j2;
      rs.v = v2;
      rs.nnz = kept;
      if (int e = phase_check("compact_a", st, sb->dbg)) return e;
    }
    mem.failed = false;
  }

  uint32_t *hist = nullptr;
  if (nhist > 0) {
    hist = mem.tmp<uint32_t>((size_t)nhist * nseg);
    if (!hist) return HS_ENOMEM;
    CK(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)nhist * nseg, st));
  }

  // the symbolic heavy rows write their sorted column lists for the numeric
  // pass into a pool of sum(min(f, n)) entries, as much of it as fits a
  // quarter of the free device memory (at most 32 GiB); rows that find no
  // room are left to the numeric pass's own bitmap build
  int32_t *glist = nullptr;
  int64_t *loff = nullptr;
  int64_t lcap = 0;
  {
    const int64_t nsh = key_off[NKEYS] - key_off[KEY_HEAVY];
    size_t free_b = 0, total_b = 0;
    if (nsh > 0 && hb->stats[3] > 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const size_t budget = free_b / 4 < ((size_t)32 << 30) ? free_b / 4 : ((size_t)32 << 30);
      const size_t want = (size_t)hb->stats[3] * 4;
      const size_t bytes = want < budget ? want : budget;
      if (bytes >= 4) {
        // (16 bytes of slack: the numeric units copy their slices in 16-byte pieces)
        glist = (int32_t *)mem.raw(bytes + 16);
        loff = glist ? (int64_t *)mem.raw(sizeof(int64_t) * (size_t)nslots) : nullptr;
        if (glist) mem.scratch.push_back({glist, bytes + 16});
        if (loff) mem.scratch.push_back({loff, sizeof(int64_t) * (size_t)nslots});
        mem.failed = false;  // optional buffers
        if (!loff) glist = nullptr;
        else {
          lcap = (int64_t)(bytes / 4);
          CK(cudaMemsetAsync(loff, 0xff, sizeof(int64_t) * (size_t)nslots, st));
        }
      }
    }
    cudaGetLastError();
  }

  // the B segment index: for every B row longer than min_len, the offset of
  // its first entry in each SEG_W-column segment (the table kept within an
  // eighth of the free memory, at most 4 GiB); built once, on first need
  int32_t *bci_id = nullptr, *bci = nullptr;
  bool bci_done = false;
  auto build_bci = [&]() -> int {
    if (bci_done || B->nnz <= 0) return HS_OK;
    bci_done = true;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const size_t budget = free_b / 8 < ((size_t)4 << 30) ? free_b / 8 : ((size_t)4 << 30);
      const int64_t stride = (int64_t)nseg + 1;
      const int64_t row_bytes = stride * 4;
      int64_t min_len = 32;
      const int64_t need = (B->nnz * row_bytes + (int64_t)budget - 1) / (int64_t)(budget ? budget : 1);
      if (need > min_len) min_len = need;
      int64_t max_rows = B->nnz / (min_len + 1);
      if (max_rows > (int64_t)(budget / row_bytes)) max_rows = (int64_t)(budget / row_bytes);
      if (max_rows > 0 && min_len < 0x7fffffff) {
        bci_id = (int32_t *)mem.raw(sizeof(int32_t) * (size_t)B->m);
        bci = bci_id ? (int32_t *)mem.raw((size_t)max_rows * (size_t)row_bytes) : nullptr;
        if (bci_id) mem.scratch.push_back({bci_id, sizeof(int32_t) * (size_t)B->m});
        if (bci) mem.scratch.push_back({bci, (size_t)max_rows * (size_t)row_bytes});
        mem.failed = false;  // optional: without it the part ends are searched
        if (!bci) bci_id = nullptr;
        else {
          PhaseTimer t("bci", st);
          launch_build_bci(rb, nseg, (int)min_len, max_rows, bci_id, bci, &sb->bci_cnt, st);
          if (int e = phase_check("bci", st, sb->dbg)) return e;
        }
      }
    }
    cudaGetLastError();
    return HS_OK;
  };

  // ---- symbolic
  SymArgs sa{rs, rb, f, nullptr, 0, Cp, hslot, hist, nseg, &sb->dyn[0], &sb->err, glist, loff, &sb->lpool, lcap};
  auto sym_bin = [&](int k0, int k1) {
    sa.list = list + key_off[k0];
    sa.count = key_off[k1] - key_off[k0];
  };
  {
    PhaseTimer t("symbolic", st);
    sym_bin(KEY_TINY, KEY_TINY + 1);
    { PhaseTimer t2("symbolic_tiny", st, sa.count > 0); launch_sym_tiny(sa, st); }
    if (int e = phase_check("symbolic_tiny", st, sb->dbg)) return e;
    sym_bin(KEY_WARP, KEY_WARP + 1);
    { PhaseTimer t2("symbolic_warp", st, sa.count > 0); launch_sym_warp(sa, st); }
    if (int e = phase_check("symbolic_warp", st, sb->dbg)) return e;
    sym_bin(KEY_MID_S, KEY_MID_S + 1);
    { PhaseTimer t2("symbolic_mid_s", st, sa.count > 0); launch_sym_mid_s(sa, st); }
    if (int e = phase_check("symbolic_mid_s", st, sb->dbg)) return e;
    sym_bin(KEY_MID, KEY_MID + 1);
    { PhaseTimer t2("symbolic_mid", st, sa.count > 0); launch_sym_mid(sa, st); }
    if (int e = phase_check("symbolic_mid", st, sb->dbg)) return e;
    sym_bin(KEY_LARGE, KEY_LARGE + 1);
    { PhaseTimer t2("symbolic_large", st, sa.count > 0); launch_sym_large(sa, st); }
    if (int e = phase_check("symbolic_large", st, sb->dbg)) return e;
    sym_bin(KEY_SPA, KEY_SPA + 1);
    { PhaseTimer t2("symbolic_spa", st, sa.count > 0); launch_sym_spa(sa, st); }
    if (int e = phase_check("symbolic_spa", st, sb->dbg)) return e;
    sym_bin(KEY_HEAVY, NKEYS);
    { PhaseTimer t2("symbolic_heavy", st, sa.count > 0); launch_sym_heavy(sa, st); }
    if (int e = phase_check("symbolic_heavy", st, sb->dbg)) return e;
  }

  // ---- offsets and numeric bins
  int64_t *scan_tmp = mem.tmp<int64_t>(scan_tmp_elems(m + 1));
  if (!scan_tmp) return HS_ENOMEM;
  {
    PhaseTimer t("scan_bin", st);
    launch_scan_i64(Cp, m + 1, scan_tmp, st);
    CK(cudaMemsetAsync(sb->key_cnt, 0, sizeof(int) * NKEYS, st));
    launch_num_count(rs, f, Cp, numeric_bins(bins, n), sb->key_cnt, st);
    launch_key_offsets(sb->key_cnt, sb->key_off, sb->key_cur, st);
    launch_scatter_num(rs, f, Cp, numeric_bins(bins, n), sb->key_cur, list, st);
    CK(cudaMemcpyAsync(&sb->nnz, Cp + m, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  }
  // numeric heavy rows that have a sorted column list run as units (column
  // parts spread over the SMs): their parts are counted now, so that the
  // number of units comes back with nnz(C); the numeric heavy rows are a
  // subset of the symbolic heavy rows, whose number bounds the count array
  int64_t *pcnt = nullptr, *pcap = nullptr;
  const int64_t nsh_rows = key_off[NKEYS] - key_off[KEY_HEAVY];
  const int ucap = unit_part_cap(vb, bins.unit_kb);
  if (glist && nsh_rows > 0) {
    pcnt = mem.tmp<int64_t>((size_t)nsh_rows);
    pcap = pcnt ? mem.tmp<int64_t>((size_t)nsh_rows) : nullptr;
    int64_t *ptmp = pcap ? mem.tmp<int64_t>((size_t)scan_tmp_elems(nsh_rows)) : nullptr;
    mem.failed = false;  // optional: without units the heavy rows run one CTA per row
    if (!ptmp) pcnt = nullptr;
    if (pcnt) {
      PhaseTimer t("scan_bin", st);
      launch_count_parts(rs, list, sb->key_off, KEY_HEAVY, hslot, hist, loff, nseg, ucap, HU_SPAN_SEGS, nsh_rows,
                         pcnt, pcap, st);
      launch_scan_i64(pcnt, nsh_rows, ptmp, st);
      launch_scan_i64(pcap, nsh_rows, ptmp, st);
      CK(cudaMemcpyAsync(&sb->nunits, pcnt + nsh_rows - 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(&sb->npcap, pcap + nsh_rows - 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    cudaGetLastError();
  }

  if (int e = phase_check("scan_bin", st, sb->dbg)) return e;
  CK(cudaMemcpyAsync(hb, sb, sizeof(SmallBlock), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hb->dbg[0]) {
    snprintf(t_detail, sizeof(t_detail), "index check %lld failed at %lld", hb->dbg[0], hb->dbg[1]);
    return HS_EINTERNAL;
  }
  if (hb->err) {
    snprintf(t_detail, sizeof(t_detail), "device consistency check %d", hb->err);
    return HS_EINTERNAL;
  }
  const int64_t nnz = hb->nnz;
  memcpy(key_off, hb->key_off, sizeof(key_off));
  C->nnz = nnz;
  if (place) {
    if (nnz > place->cap) return HS_ECAPACITY;
    C->idx = place->idx;
    C->val = vb ? place->val : nullptr;
  } else {
    C->idx = (int32_t *)outmem.raw(sizeof(int32_t) * (size_t)nnz);
    if (!C->idx) return HS_ENOMEM;
    if (vb) {
      C->val = outmem.raw((size_t)vb * (size_t)nnz);
      if (!C->val) return HS_ENOMEM;
    }
  }

  // ---- numeric
  // heavy bin: units, planned from the segment counts of the rows with lists
  // and, for semirings with values, each unit's B segments (start, product
  // prefix, left value) laid out by launch_build_pairs once the segment
  // index exists (below)
  HeavyUnit *units = nullptr;
  int64_t *pstart = nullptr;
  int32_t *ppre = nullptr;
  void *paval = nullptr;
  const int64_t nunits = pcnt ? hb->nunits : 0;
  const int64_t npcap = pcnt ? hb->npcap : 0;
  const int nheavy = key_off[NKEYS] - key_off[KEY_HEAVY];
  const int a_bytes = (sr == HS_PLUS_TIMES || sr == HS_MIN_PLUS || sr == HS_SELECT1ST) ? vb : 0;
  if (nheavy > 0 && nunits > 0) {
    units = mem.tmp<HeavyUnit>((size_t)nunits);
    if (units && vb) {  // 16 bytes of slack each: the units copy their slices in 16-byte pieces
      pstart = (int64_t *)mem.tmp<char>((size_t)npcap * 8 + 16);
      ppre = (int32_t *)mem.tmp<char>((size_t)npcap * 4 + 16);
      paval = a_bytes ? (void *)mem.tmp<char>((size_t)npcap * a_bytes + 16) : nullptr;
      if (!pstart || !ppre || (a_bytes && !paval)) units = nullptr;
    }
    mem.failed = false;  // optional, as above
    if (units) {
      PhaseTimer t("scan_bin", st);
      launch_plan_parts(rs, list + key_off[KEY_HEAVY], nheavy, hslot, hist, loff, Cp, nseg, ucap, HU_SPAN_SEGS,
                        pcnt, pcap, units, st);
    }
    cudaGetLastError();
  }
  // rows that a unit does not cover (no list): one CTA per row, with
  // per-A-entry cursors into B rows (relative offsets)
  const bool lists_partial = lcap < (int64_t)hb->stats[3];
  int32_t *gcur = nullptr, *gend = nullptr;
  if (nheavy > 0 && (!units || lists_partial)) {
    gcur = mem.tmp<int32_t>((size_t)A->nnz);
    gend = mem.tmp<int32_t>((size_t)A->nnz);
    if (!gcur || !gend) return HS_ENOMEM;
  }
  // heavy bin: the B segment index (built before the symbolic pass when
  // symbolic units used it)
  if (key_off[NKEYS] > key_off[KEY_HEAVY])
    if (int e = build_bci()) return e;
  if (units && vb) {
    PhaseTimer t("heavy_pairs", st);
    launch_build_pairs(rs, rb, units, nunits, bci_id, bci, nseg, a_bytes, pstart, ppre, paval, st);
    if (int e = phase_check("heavy_pairs", st, sb->dbg)) return e;
  }
  NumArgs na{rs, rb,   f,    nullptr, 0,    Cp,    C->idx, C->val, hslot,
             hist, nseg, &sb->dyn[1], &sb->err, gcur, gend, glist, loff, bci_id, bci};
  na.unsorted = (flags & HS_FLAG_UNSORTED) ? 1 : 0;
  na.units = units;
  na.nunits = units ? nunits : 0;
  na.udyn = &sb->dyn[2];
  na.lists_partial = lists_partial ? 1 : 0;
  na.pstart = pstart;
  na.ppre = ppre;
  na.paval = paval;
  na.pair_abytes = a_bytes;
  na.unit_kb = bins.unit_kb;
  const char *names[NUM_KINDS] = {"numeric_tiny",   "numeric_warp_s", "numeric_warp",   "numeric_mid_s",
                                  "numeric_mid",    "numeric_large_s", "numeric_large", "numeric_sort_xs",
                                  "numeric_sort_s", "numeric_sort_m",  "numeric_sort",  "numeric_spa",
                                  "numeric_heavy"};
  static_assert(KEY_TINY + NUM_KINDS - 1 == KEY_HEAVY, "one key per numeric kind before the heavy keys");
  {
    PhaseTimer t("numeric", st);
    for (int kind = 0; kind < NUM_KINDS; ++kind) {
      const int k0 = KEY_TINY + kind, k1 = kind == NUM_KINDS - 1 ? NKEYS : k0 + 1;
      na.list = list + key_off[k0];
      na.count = key_off[k1] - key_off[k0];
      if (plan) {
        plan->off[kind] = key_off[k0];
        plan->count[kind] = na.count;
      }
      {
        PhaseTimer t2(names[kind], st, na.count > 0);
        if (na.count > 0 && !launch_num(sr, out_dt, kind, na, st)) return HS_EINVAL;
      }
      if (int e = phase_check(names[kind], st, sb->dbg)) return e;
    }
  }
  if (flags & HS_FLAG_VALIDATE) {
    CK(cudaMemcpyAsync(hb, sb, sizeof(SmallBlock), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hb->dbg[0]) {
      snprintf(t_detail, sizeof(t_detail), "index check %lld failed at %lld", hb->dbg[0], hb->dbg[1]);
      return HS_EINTERNAL;
    }
    if (hb->err) {
      snprintf(t_detail, sizeof(t_detail), "device consistency check %d", hb->err);
      return HS_EINTERNAL;
    }
  }
  // explicit zeros on request: entries whose (+,x) sum is exactly zero are
  // removed by one compaction of C (the symbolic pass counts structure only,
  // so this cannot happen earlier)
  if ((flags & HS_FLAG_PRUNE_ZEROS) && sr == HS_PLUS_TIMES && !plan && !place && nnz > 0) {
    int64_t *keep = mem.tmp<int64_t>((size_t)nnz);
    int64_t *ktmp = mem.tmp<int64_t>((size_t)scan_tmp_elems(nnz));
    if (mem.failed) return HS_ENOMEM;
    {
      PhaseTimer t("prune_zeros", st);
      launch_keep_nonzero(C->val, out_dt, nnz, keep, st);
      launch_scan_i64(keep, nnz, ktmp, st);
    }
    CK(cudaMemcpyAsync(&hb->nnz, keep + nnz - 1, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int64_t kept = hb->nnz;
    if (kept < nnz) {
      int64_t *p2 = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(m + 1));
      int32_t *j2 = (int32_t *)outmem.raw(sizeof(int32_t) * (size_t)(kept > 0 ? kept : 1));
      void *v2 = outmem.raw((size_t)vb * (size_t)(kept > 0 ? kept : 1));
      if (!p2 || !j2 || !v2) {
        if (p2) outmem.release(p2, sizeof(int64_t) * (size_t)(m + 1));
        if (j2) outmem.release(j2, sizeof(int32_t) * (size_t)(kept > 0 ? kept : 1));
        if (v2) outmem.release(v2, (size_t)vb * (size_t)(kept > 0 ? kept : 1));
        return HS_ENOMEM;
      }
      const RowSet cs{Cp, C->idx, C->val, nullptr, m, nnz, m, sb->dbg};
      {
        PhaseTimer t("prune_zeros", st);
        launch_compact_by_keep(cs, keep, j2, v2, vb, p2, st);
      }
      outmem.release(C->ptr, sizeof(int64_t) * (size_t)(m + 1));
      outmem.release(C->idx, sizeof(int32_t) * (size_t)nnz);
      outmem.release(C->val, (size_t)vb * (size_t)nnz);
      C->ptr = p2;
      C->idx = j2;
      C->val = v2;
      C->nnz = kept;
    }
    if (int e = check_launch()) return e;
  }
  if (plan) {  // the plan takes over every scratch buffer
    plan->c_nnz = nnz;
    plan->na = na;
    plan->list = list;
    plan->dyn = &sb->dyn[1];
    plan->err = &sb->err;
    plan->dbg = sb->dbg;
    plan->blocks = std::move(mem.scratch);
    mem.scratch.clear();
  }
  return HS_OK;
}

// runs fn; on failure releases whatever fn allocated for C
template <class F> static int with_output(hs_mat *C, Mem &outmem, F &&fn) {
  int e = fn();
  if (e != HS_OK && C) free_mat(C, outmem);
  return e;
}

static int sparse_impl(const int32_t *I, const int32_t *J, const void *V, int64_t nnz, int64_t m, int64_t n,
                       int dtype, int sr, hs_mat *C, Mem &mem, Mem &outmem, uint32_t flags);

// B = A(I, J) (Section 3.1's SpRef), the triple product R*A*Q evaluated
// without forming R*A: the rows I[t] are gathered end to end, each gathered
// entry (t, c, v) yields (t, p, v) for every p with J[p] == c (Q's row c),
// and the tuples are ordered by (t, p) with the radix sort of sparse(); when
// J is strictly increasing they are in order already and are written out
// directly.  Four host synchronisations (three with a strictly increasing J).
static int spref_impl(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ, hs_mat *Bout,
                      Mem &mem, Mem &outmem, uint32_t flags) {
  cudaStream_t st = mem.st;
  if (!A || !Bout || A->fmt != HS_CSR || nI < 0 || nJ < 0) return HS_EINVAL;
  if ((nI > 0 && !I) || (nJ > 0 && !J)) return HS_EINVAL;
  if (nI > 0x7fffffffLL || nJ > 0x7fffffffLL) return HS_EUNSUPPORTED;
  if (!dtype_ok(A->dtype) || (A->m > 0 && !A->ptr)) return HS_EINVAL;
  if (A->dtype != HS_BOOL && A->nnz > 0 && !A->val) return HS_EINVAL;
  const int vb = A->dtype == HS_BOOL ? 0 : vbytes_of(A->dtype);
  const int64_t n = A->n;
  int *flag = mem.tmp<int>(2);
  unsigned long long *qmax = mem.tmp<unsigned long long>(1);
  int64_t *hbuf = (int64_t *)pinned(32);
  int64_t *Qp = mem.tmp<int64_t>(n + 1);
  int64_t *Qcur = mem.tmp<int64_t>(n + 1);
  int32_t *Qj = mem.tmp<int32_t>(nJ > 0 ? nJ : 1);
  int64_t *G = mem.tmp<int64_t>(nI + 1);
  int64_t *scan_tmp = mem.tmp<int64_t>(scan_tmp_elems((n + 1) > (nI + 1) ? (n + 1) : (nI + 1)));
  if (mem.failed || !hbuf) return HS_ENOMEM;
  // index ranges are always checked, and before any kernel uses I or J as
  // an address: they index A's rows, Q's rows and the gathered offsets (the
  // row counts of Q skip out-of-range ids, so they run alongside)
  CK(cudaMemsetAsync(flag, 0, 8, st));
  CK(cudaMemsetAsync(qmax, 0, 8, st));
  CK(cudaMemsetAsync(Qp, 0, sizeof(int64_t) * (size_t)(n + 1), st));
  launch_check_range(I, nI, A->m, flag, st);
  launch_check_range(J, nJ, n, flag, st);
  launch_check_increasing(J, nJ, flag, st);
  if (flags & HS_FLAG_VALIDATE) launch_validate(A->ptr, A->idx, A->m, A->n, flag + 1, st);
  launch_build_Q_count(J, nJ, n, Qp, st);
  launch_max_count(Qp, n + 1, qmax, st);
  CK(cudaMemcpyAsync(hbuf, flag, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hbuf + 1, qmax, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int fl = ((int *)hbuf)[0], vf = ((int *)hbuf)[1];
  if (fl & 1) return HS_EINVAL;
  if (vf & 5) return HS_EINVAL;
  if (vf & 2) return HS_ENONCANON;
  const bool increasing = !(fl & 4);
  const int64_t qrow_max = hbuf[1];
  // Q = sparse(J, 1:len(J), 1, n, len(J)): row k holds every p with J[p] == k,
  // increasing.  Short rows (at most 32 repetitions of an index): counted,
  // filled by atomics and sorted in place; otherwise built by the stable
  // radix sort of sparse() itself
  struct QGuard {
    hs_mat q{};
    Mem &m;
    ~QGuard() { free_mat(&q, m); }
  } qg{hs_mat{}, mem};
  if (qrow_max <= 32) {
    PhaseTimer t("spref_build", st);
    launch_scan_i64(Qp, n + 1, scan_tmp, st);
    CK(cudaMemcpyAsync(Qcur, Qp, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, st));
    launch_build_Q_fill(J, nJ, Qcur, Qj, st);
    launch_sort_short_rows(Qp, Qj, n, st);
  } else {
    int32_t *pidx = mem.tmp<int32_t>((size_t)nJ);
    if (!pidx) return HS_ENOMEM;
    launch_iota_i32(pidx, nJ, st);
    if (int e = sparse_impl(J, pidx, nullptr, nJ, n, nJ, HS_BOOL, HS_OR_AND, &qg.q, mem, mem, 0)) return e;
    Qp = qg.q.ptr;
    Qj = qg.q.idx;
  }
  {
    PhaseTimer t("spref_gather", st);
    CK(cudaMemsetAsync(G, 0, sizeof(int64_t) * (size_t)(nI + 1), st));
    launch_gather_len(A->ptr, I, nI, G, st);
    launch_scan_i64(G, nI + 1, scan_tmp, st);
  }
  CK(cudaMemcpyAsync(hbuf, G + nI, 8, cudaMemcpyDeviceToHost, st));
  if (int e = check_launch()) return e;
  CK(cudaStreamSynchronize(st));
  const int64_t total = hbuf[0];

  auto empty_out = [&]() {
    memset(Bout, 0, sizeof(*Bout));
    Bout->fmt = HS_CSR;
    Bout->dtype = A->dtype;
    Bout->m = nI;
    Bout->n = nJ;
    Bout->ptr = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(nI + 1));
    Bout->idx = (int32_t *)outmem.raw(4);
    Bout->val = vb ? outmem.raw((size_t)vb) : nullptr;
    if (!Bout->ptr || !Bout->idx || (vb && !Bout->val)) return HS_ENOMEM;
    CK(cudaMemsetAsync(Bout->ptr, 0, sizeof(int64_t) * (size_t)(nI + 1), st));
    return check_launch();
  };
  if (total == 0 || nJ == 0) return empty_out();

  int64_t *inc = mem.tmp<int64_t>((size_t)total);
  int64_t *W = mem.tmp<int64_t>((size_t)total);
  int64_t *scan_g = mem.tmp<int64_t>(scan_tmp_elems(total));
  if (mem.failed) return HS_ENOMEM;
  GatherArgs ga{A->ptr, A->idx, A->val, vb, I, G, inc, Qp, Qj, total, n};
  {
    PhaseTimer t("spref_gather", st);
    CK(cudaMemsetAsync(inc, 0, sizeof(int64_t) * (size_t)total, st));
    launch_row_starts(G, nI, total, inc, st);
    launch_scan_i64(inc, total, scan_g, st);
    launch_gather_w(ga, W, st);
    launch_scan_i64(W, total, scan_g, st);
  }
  CK(cudaMemcpyAsync(hbuf, W + total - 1, 8, cudaMemcpyDeviceToHost, st));
  if (int e = check_launch()) return e;
  CK(cudaStreamSynchronize(st));
  const int64_t ntup = hbuf[0];
  if (ntup == 0) return empty_out();

  if (increasing) {
    memset(Bout, 0, sizeof(*Bout));
    Bout->fmt = HS_CSR;
    Bout->dtype = A->dtype;
    Bout->m = nI;
    Bout->n = nJ;
    Bout->nnz = ntup;
    Bout->ptr = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(nI + 1));
    Bout->idx = (int32_t *)outmem.raw(sizeof(int32_t) * (size_t)ntup);
    Bout->val = vb ? outmem.raw((size_t)vb * (size_t)ntup) : nullptr;
    if (!Bout->ptr || !Bout->idx || (vb && !Bout->val)) return HS_ENOMEM;
    PhaseTimer t("spref_emit", st);
    launch_gather_offsets(G, nI, W, Bout->ptr, st);
    launch_gather_direct(ga, W, Bout->idx, Bout->val, st);
    return check_launch();
  }
  if (ntup > 0x7fffffffLL) return HS_EUNSUPPORTED;
  int32_t *ti = mem.tmp<int32_t>((size_t)ntup);
  int32_t *pj = mem.tmp<int32_t>((size_t)ntup);
  void *tv = vb ? (void *)mem.tmp<char>((size_t)vb * (size_t)ntup) : nullptr;
  if (mem.failed) return HS_ENOMEM;
  {
    PhaseTimer t("spref_gather", st);
    launch_gather_fill(ga, W, ti, pj, tv, st);
  }
  if (int e = check_launch()) return e;
  // every (t, p) occurs once, so the combining operation never acts: values
  // are copied bit for bit whatever the operation
  const int sr = A->dtype == HS_BOOL ? HS_OR_AND : A->dtype == HS_I32 ? HS_MIN_PLUS : HS_PLUS_TIMES;
  return sparse_impl(ti, pj, tv, ntup, nI, nJ, A->dtype, sr, Bout, mem, outmem, flags);
}

// C = sparse(i, j, v, m, n) (Section 2's constructor).  Every tuple is the
// key (i << bits(n-1)) | j, so that ascending keys are CSR order; a stable
// radix sort of the keys, carrying v, puts the tuples of one position next to
// each other in input order, and each run of equal keys becomes one entry of
// C, its values folded with the semiring's add (kernels in sparse.cu).  One
// host synchronisation: after the sort, to learn nnz(C) and whether an index
// was out of range.
static int bits_of(int64_t x) { return x > 0 ? 64 - __builtin_clzll((unsigned long long)x) : 0; }

// Failure-detection test setting for the next sparse() sort on this host
// thread (hs_test_lookback_expiry): a short look-back poll limit and a tile
// that never publishes its counts.  Consumed by one call.
static thread_local int t_sp_spin = 0;             // 0: the production limit
static thread_local long long t_sp_withhold = -1;  // -1: every tile publishes

static int sparse_impl(const int32_t *I, const int32_t *J, const void *V, int64_t nnz, int64_t m, int64_t n,
                       int dtype, int sr, hs_mat *C, Mem &mem, Mem &outmem, uint32_t) {
  cudaStream_t st = mem.st;
  if (!C || nnz < 0 || m < 0 || n < 0) return HS_EINVAL;
  int op = -1;
  if (sr == HS_PLUS_TIMES) op = dtype == HS_F64 ? 0 : dtype == HS_F32 ? 1 : dtype == HS_I64 ? 2 : -1;
  else if (sr == HS_MIN_PLUS) op = dtype == HS_F32 ? 3 : dtype == HS_I32 ? 4 : -1;
  else if (sr == HS_OR_AND) op = dtype == HS_BOOL ? 5 : -1;
  if (op < 0) return HS_EINVAL;
  if (nnz > 0 && (!I || !J || (dtype != HS_BOOL && !V))) return HS_EINVAL;
  if (nnz > 0x7fffffffLL || m > 0x7fffffffLL || n > 0x7fffffffLL) return HS_EUNSUPPORTED;
  const int vb = vbytes_of(dtype);
  memset(C, 0, sizeof(*C));
  C->fmt = HS_CSR;
  C->dtype = dtype;
  C->m = m;
  C->n = n;
  C->ptr = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(m + 1));
  if (!C->ptr) return HS_ENOMEM;
  CK(cudaMemsetAsync(C->ptr, 0, sizeof(int64_t) * (size_t)(m + 1), st));
  if (nnz == 0) {
    C->idx = (int32_t *)outmem.raw(4);
    C->val = vb ? outmem.raw((size_t)vb) : nullptr;
    if (!C->idx || (vb && !C->val)) return HS_ENOMEM;
    return check_launch();
  }
  const int nbj = bits_of(n - 1), nbi = bits_of(m - 1);
  const int rb = sp_radix_bits();
  int passes = (nbi + nbj + rb - 1) / rb;
  if (passes < 1) passes = 1;
  if (passes > sp_max_passes()) return HS_EINTERNAL;
  const int64_t tiles = sp_tiles(nnz);
  const int64_t longcap = sp_long_capacity(nnz);
  const int64_t scan_n = tiles > m + 1 ? tiles : m + 1;
  uint64_t *kbuf[2] = {mem.tmp<uint64_t>((size_t)nnz), mem.tmp<uint64_t>((size_t)nnz)};
  void *vbuf[2] = {nullptr, nullptr};
  if (vb) {
    vbuf[0] = mem.tmp<char>((size_t)nnz * vb);
    vbuf[1] = mem.tmp<char>((size_t)nnz * vb);
  }
  unsigned long long *status = mem.tmp<unsigned long long>((size_t)(tiles << rb));
  unsigned long long *ghist = mem.tmp<unsigned long long>((size_t)passes << rb);
  int *ticket = mem.tmp<int>((size_t)passes);
  int64_t *theads = mem.tmp<int64_t>((size_t)tiles);
  int64_t *scan_tmp = mem.tmp<int64_t>((size_t)scan_tmp_elems(scan_n));
  int64_t *longlist = vb ? mem.tmp<int64_t>((size_t)(2 * longcap)) : nullptr;
  int *flags = mem.tmp<int>(2);  // [0] index out of range, [1] long runs
  int64_t *host = (int64_t *)pinned(16);
  if (mem.failed || !host) return HS_ENOMEM;
  CK(cudaMemsetAsync(flags, 0, 8, st));
  CK(cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)(tiles << rb), st));
  CK(cudaMemsetAsync(ghist, 0, sizeof(unsigned long long) * ((size_t)passes << rb), st));
  CK(cudaMemsetAsync(ticket, 0, sizeof(int) * (size_t)passes, st));
  int cur = 0;
  const int spin = t_sp_spin > 0 ? t_sp_spin : sp_spin_limit();
  const long long withhold = t_sp_withhold;
  t_sp_spin = 0;
  t_sp_withhold = -1;
  {
    PhaseTimer t("sparse_sort", st);
    launch_sp_allhist(I, J, nnz, nbj, m, n, passes, ghist, flags, st);
    for (int p = 0; p < passes; ++p) {
      const bool first = p == 0;
      const uint64_t *kin = first ? nullptr : kbuf[cur];
      const void *vin = first ? V : vbuf[cur];
      const int out = first ? 0 : cur ^ 1;
      PhaseTimer tp("sparse_pass", st);
      launch_sp_pass(vb, kin, I, J, vin, nnz, nbj, m, n, p, ghist + ((size_t)p << rb), status, ticket + p, tiles,
                     kbuf[out], vbuf[out], flags, spin, withhold, st);
      cur = out;
    }
    launch_sp_heads(kbuf[cur], nnz, theads, tiles, st);
    launch_scan_i64(theads, tiles, scan_tmp, st);
  }
  if (int e = check_launch()) return e;
  CK(cudaMemcpyAsync(host, theads + tiles - 1, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(host + 1, flags, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int fl = *(int *)(host + 1);
  if (fl & 1) return HS_EINVAL;
  if (fl & 2) return HS_ETIMEDOUT;
  const int64_t U = host[0];
  C->nnz = U;
  C->idx = (int32_t *)outmem.raw(sizeof(int32_t) * (size_t)U);
  C->val = vb ? outmem.raw((size_t)vb * (size_t)U) : nullptr;
  if (!C->idx || (vb && !C->val)) return HS_ENOMEM;
  {
    PhaseTimer t("sparse_emit", st);
    launch_sp_emit(op, kbuf[cur], vbuf[cur], nnz, nbj, theads, tiles, C->idx, C->val, C->ptr, longlist,
                   flags + 1, st);
    launch_scan_i64(C->ptr, m + 1, scan_tmp, st);
  }
  return check_launch();
}

static int spasgn_impl(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ,
                       const hs_mat *B, int accumulate, int add_sr, hs_mat *C, Mem &mem, Mem &outmem,
                       uint32_t flags) {
  cudaStream_t st = mem.st;
  if (!A || !B || !C || A->fmt != HS_CSR || B->fmt != HS_CSR) return HS_EINVAL;
  if (nI < 0 || nJ < 0 || B->m != nI || B->n != nJ || A->dtype != B->dtype) return HS_EINVAL;
  if ((nI > 0 && !I) || (nJ > 0 && !J)) return HS_EINVAL;
  if (accumulate && A->dtype != HS_BOOL && add_sr != HS_PLUS_TIMES && add_sr != HS_MIN_PLUS) return HS_EINVAL;
  const int vb = vbytes_of(A->dtype);
  const int64_t m = A->m, n = A->n;
  int32_t *rpos = mem.tmp<int32_t>(m > 0 ? m : 1);
  int32_t *cpos = mem.tmp<int32_t>(n > 0 ? n : 1);
  int *flag = mem.tmp<int>(2);
  int *hflag = (int *)pinned(8);
  if (mem.failed || !hflag) return HS_ENOMEM;
  CK(cudaMemsetAsync(flag, 0, 8, st));
  launch_fill_i32(rpos, m, -1, st);
  launch_fill_i32(cpos, n, -1, st);
  launch_mark_positions(I, nI, m, rpos, flag, st);
  launch_mark_positions(J, nJ, n, cpos, flag, st);
  CK(cudaMemcpyAsync(hflag, flag, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hflag[0] & 1) return HS_EINVAL;
  if (hflag[0] & 2) return HS_EDUP;

  // R = sparse(I, 1:mb, 1, ma, mb) and Q = sparse(1:nb, J, 1, nb, na)
  int64_t *Rp = mem.tmp<int64_t>(m + 1);
  int32_t *Rj = mem.tmp<int32_t>(nI > 0 ? nI : 1);
  int64_t *Qp = mem.tmp<int64_t>(nJ + 1);
  int64_t *scan_tmp = mem.tmp<int64_t>(scan_tmp_elems((m > n ? m : n) + 1));
  if (mem.failed) return HS_ENOMEM;
  {
    PhaseTimer t("spasgn_build", st);
    CK(cudaMemsetAsync(Rp, 0, sizeof(int64_t), st));
    launch_rows_from_pos(rpos, m, Rp, st);
    launch_scan_i64(Rp, m + 1, scan_tmp, st);
    launch_fill_from_pos(rpos, m, Rp, Rj, st);
    launch_iota_i64(Qp, nJ + 1, st);
  }
  hs_mat R{HS_CSR, HS_BOOL, m, nI, nI, 0, Rp, Rj, nullptr, nullptr};
  hs_mat Q{HS_CSR, HS_BOOL, nJ, n, nJ, 0, Qp, const_cast<int32_t *>(J), nullptr, nullptr};
  hs_mat RB, X;
  memset(&RB, 0, sizeof(RB));
  memset(&X, 0, sizeof(X));
  // the products feed the merge, which needs canonical rows
  const uint32_t pf = flags & ~(HS_FLAG_VALIDATE | HS_FLAG_UNSORTED | HS_FLAG_PRUNE_ZEROS);
  int e = spgemm_impl(HS_SELECT2ND, &R, B, &RB, mem, mem, pf);
  if (!e) e = spgemm_impl(HS_SELECT1ST, &RB, &Q, &X, mem, mem, pf);
  free_mat(&RB, mem);
  if (e) {
    free_mat(&X, mem);
    return e;
  }
  // C = A .* not(S*A*T) + R*B*Q  (or A + R*B*Q for extend-add)
  memset(C, 0, sizeof(*C));
  C->fmt = HS_CSR;
  C->dtype = A->dtype;
  C->m = m;
  C->n = n;
  C->ptr = (int64_t *)outmem.raw(sizeof(int64_t) * (size_t)(m + 1));
  if (!C->ptr) {
    free_mat(&X, mem);
    return HS_ENOMEM;
  }
  AsgnArgs aa{A->ptr, A->idx, A->val, X.ptr, X.idx, X.val, rpos, cpos, m, vb, accumulate, add_sr, A->dtype,
              C->ptr, nullptr, nullptr};
  int64_t *hnnz = (int64_t *)pinned(8);
  {
    PhaseTimer t("spasgn_merge", st);
    CK(cudaMemsetAsync(C->ptr, 0, sizeof(int64_t), st));
    launch_asgn_count(aa, st);
    launch_scan_i64(C->ptr, m + 1, scan_tmp, st);
  }
  CK(cudaMemcpyAsync(hnnz, C->ptr + m, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  C->nnz = *hnnz;
  C->idx = (int32_t *)outmem.raw(sizeof(int32_t) * (size_t)C->nnz);
  if (vb) C->val = outmem.raw((size_t)vb * (size_t)C->nnz);
  if (!C->idx || (vb && !C->val)) {
    free_mat(&X, mem);
    return HS_ENOMEM;
  }
  aa.Cj = C->idx;
  aa.Cv = C->val;
  {
    PhaseTimer t("spasgn_merge", st);
    launch_asgn_fill(aa, st);
  }
  free_mat(&X, mem);
  return check_launch();
}

}  // namespace hs

using namespace hs;

extern "C" {

int hs_spgemm(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C, const hs_allocator *al, void *stream,
              uint32_t flags) {
  if (!C) return HS_EINVAL;
  memset(C, 0, sizeof(*C));
  t_detail[0] = 0;
  Mem mem{al, (cudaStream_t)stream};
  Mem out{al, (cudaStream_t)stream};
  return with_output(C, out, [&] { return spgemm_impl(semiring, A, B, C, mem, out, flags); });
}

int hs_plan_create(int semiring, const hs_mat *A, const hs_mat *B, hs_mat *C, hs_plan **plan,
                   const hs_allocator *al, void *stream, uint32_t flags) {
  if (!C || !plan) return HS_EINVAL;
  memset(C, 0, sizeof(*C));
  *plan = nullptr;
  t_detail[0] = 0;
  hs_plan *P = new (std::nothrow) hs_plan();
  if (!P) return HS_ENOMEM;
  Mem mem{al, (cudaStream_t)stream};
  Mem out{al, (cudaStream_t)stream};
  const int e = with_output(C, out, [&] { return spgemm_impl(semiring, A, B, C, mem, out, flags, P); });
  if (e != HS_OK) {
    for (auto &b : P->blocks) mem.release(b.p, b.n);
    delete P;
    return e;
  }
  if (al) {
    P->al = *al;
    P->has_al = true;
  }
  *plan = P;
  return HS_OK;
}

int hs_plan_execute(const hs_plan *P, const void *A_val, const void *B_val, void *C_val, void *stream) {
  if (!P) return HS_EINVAL;
  const int vb = vbytes_of(P->out_dt);
  const bool need_a = P->sr == HS_PLUS_TIMES || P->sr == HS_MIN_PLUS || (P->sr == HS_SELECT1ST && vb);
  const bool need_b = P->sr == HS_PLUS_TIMES || P->sr == HS_MIN_PLUS || (P->sr == HS_SELECT2ND && vb);
  if ((need_a && P->a_nnz && !A_val) || (need_b && P->b_nnz && !B_val) || (vb && P->c_nnz && !C_val))
    return HS_EINVAL;
  if (P->c_nnz == 0) return HS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  NumArgs na = P->na;
  na.A.v = A_val;
  na.B.v = B_val;
  na.Cv = C_val;
  CK(cudaMemsetAsync(P->dyn, 0, 2 * sizeof(int), st));  // the heavy rows' and units' counters
  // the heavy units' B segments carry A's values: laid out again from the new ones
  if (na.units && na.pstart && na.nunits > 0)
    launch_build_pairs(na.A, na.B, const_cast<HeavyUnit *>(na.units), na.nunits, na.bci_id, na.bci, na.nseg,
                       na.pair_abytes, const_cast<int64_t *>(na.pstart), const_cast<int32_t *>(na.ppre),
                       const_cast<void *>(na.paval), st);
  for (int kind = 0; kind < NUM_KINDS; ++kind) {
    if (P->count[kind] <= 0) continue;
    na.list = P->list + P->off[kind];
    na.count = P->count[kind];
    if (!launch_num(P->sr, P->out_dt, kind, na, st)) return HS_EINVAL;
  }
  return check_launch();
}

int hs_plan_status(const hs_plan *P, void *stream) {
  if (!P) return HS_EINVAL;
  if (!P->err) return HS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int *h = (int *)pinned(3 * sizeof(long long));
  if (!h) return HS_ECUDA;
  long long *hd = reinterpret_cast<long long *>(h) + 1;
  CK(cudaMemcpyAsync(h, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hd, P->dbg, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hd[0]) {
    snprintf(t_detail, sizeof(t_detail), "index check %lld failed at %lld", hd[0], hd[1]);
    return HS_EINTERNAL;
  }
  if (h[0]) {
    snprintf(t_detail, sizeof(t_detail), "device consistency check %d", h[0]);
    return HS_EINTERNAL;
  }
  return HS_OK;
}

void hs_plan_destroy(hs_plan *P, void *stream) {
  if (!P) return;
  Mem mem{P->has_al ? &P->al : nullptr, (cudaStream_t)stream};
  for (auto &b : P->blocks) mem.release(b.p, b.n);
  P->blocks.clear();
  delete P;
}

int hs_spgemm_to_host(int semiring, const hs_mat *A, const hs_mat *B, int64_t nblocks, int64_t *h_ptr,
                      int32_t *h_idx, void *h_val, int64_t capacity, int64_t *nnz_out, void *stream,
                      uint32_t flags) {
  if (!A || !B || !h_ptr || !nnz_out || nblocks < 1 || capacity < 0) return HS_EINVAL;
  if (A->fmt != HS_CSR || A->m < 0) return HS_EINVAL;
  int out_dt = 0;
  if (!numeric_supported(semiring, A->dtype, B->dtype, out_dt)) return HS_EINVAL;
  const int vb = vbytes_of(out_dt);
  if ((capacity > 0 && !h_idx) || (vb && capacity > 0 && !h_val)) return HS_EINVAL;
  *nnz_out = 0;
  t_detail[0] = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStream_t cs = nullptr;  // copies of finished blocks run here, beside the next block's product
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return HS_ECUDA;
  }
  cudaMemPool_t pool = own_pool();
  const int64_t m = A->m;
  // Host arrays that the GPU maps (page-locked memory under unified
  // addressing; on NVLink-C2C systems the stores travel while the kernels
  // run): the numeric kernels write C's columns and values there directly,
  // so nothing is copied afterwards but the row offsets.
  auto mapped = [](const void *h) -> void * {
    if (!h) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
  };
  int32_t *d_idx = (int32_t *)mapped(h_idx);
  void *d_val = vb ? mapped(h_val) : nullptr;
  if (nblocks == 1 && capacity > 0 && d_idx && (!vb || d_val) && !(flags & HS_FLAG_STAGE_ON_DEVICE)) {
    hs_mat Cd;
    memset(&Cd, 0, sizeof(Cd));
    Mem mem{nullptr, st, pool};
    Mem out{nullptr, st, pool};
    const OutPlace place{d_idx, d_val, capacity};
    int status = spgemm_impl(semiring, A, B, &Cd, mem, out, flags, nullptr, &place);
    *nnz_out = Cd.nnz;
    if (status == HS_OK) {
      if (cudaMemcpyAsync(h_ptr, Cd.ptr, sizeof(int64_t) * (size_t)(m + 1), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        status = HS_ECUDA;
      }
    }
    if (Cd.ptr) out.release(Cd.ptr, sizeof(int64_t) * (size_t)(m + 1));
    cudaEventDestroy(ev);
    cudaStreamDestroy(cs);
    return status;
  }
  const int64_t rows_per = (m + nblocks - 1) / nblocks;
  int64_t base = 0;
  int status = HS_OK;
  for (int64_t r0 = 0; r0 < m || (m == 0 && r0 == 0); r0 += (rows_per ? rows_per : 1)) {
    const int64_t r1 = m == 0 ? 0 : (r0 + rows_per < m ? r0 + rows_per : m);
    // rows r0..r1 of A as a matrix of their own (offsets stay absolute)
    hs_mat Ab = *A;
    Ab.m = r1 - r0;
    Ab.ptr = A->ptr + r0;
    hs_mat Cb;
    memset(&Cb, 0, sizeof(Cb));
    Mem mem{nullptr, st, pool};
    Mem out{nullptr, st, pool};
    status = with_output(&Cb, out,
                         [&] { return spgemm_impl(semiring, &Ab, B, &Cb, mem, out, flags & ~HS_FLAG_PRUNE_ZEROS); });
    if (status != HS_OK) break;
    const int64_t rows = r1 - r0;
    if (base + Cb.nnz <= capacity) {
      if (base) launch_add_i64(Cb.ptr, rows + 1, base, st);
      if (cudaEventRecord(ev, st) != cudaSuccess || cudaStreamWaitEvent(cs, ev, 0) != cudaSuccess ||
          cudaMemcpyAsync(h_ptr + r0, Cb.ptr, sizeof(int64_t) * (size_t)(rows + 1), cudaMemcpyDeviceToHost, cs) !=
              cudaSuccess ||
          (Cb.nnz && cudaMemcpyAsync(h_idx + base, Cb.idx, sizeof(int32_t) * (size_t)Cb.nnz,
                                     cudaMemcpyDeviceToHost, cs) != cudaSuccess) ||
          (vb && Cb.nnz &&
           cudaMemcpyAsync(reinterpret_cast<char *>(h_val) + (size_t)base * vb, Cb.val, (size_t)vb * (size_t)Cb.nnz,
                           cudaMemcpyDeviceToHost, cs) != cudaSuccess)) {
        cudaGetLastError();
        status = HS_ECUDA;
      }
    } else if (cudaEventRecord(ev, st) != cudaSuccess || cudaStreamWaitEvent(cs, ev, 0) != cudaSuccess) {
      cudaGetLastError();
      status = HS_ECUDA;
    }
    // the block's output goes back to the pool on the copy stream, after its copies
    cudaFreeAsync(Cb.ptr, cs);
    cudaFreeAsync(Cb.idx, cs);
    if (Cb.val) cudaFreeAsync(Cb.val, cs);
    base += Cb.nnz;
    if (status != HS_OK || m == 0) break;
  }
  if (cudaStreamSynchronize(cs) != cudaSuccess && status == HS_OK) {
    cudaGetLastError();
    status = HS_ECUDA;
  }
  cudaEventDestroy(ev);
  cudaStreamDestroy(cs);
  *nnz_out = base;
  if (status == HS_OK && base > capacity) status = HS_ECAPACITY;
  return status;
}

int hs_trim_memory(void) {
  cudaMemPool_t pool = own_pool();
  if (!pool) return HS_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return HS_ECUDA;
  }
  return HS_OK;
}

int hs_spref(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ, hs_mat *B,
             const hs_allocator *al, void *stream, uint32_t flags) {
  if (!B) return HS_EINVAL;
  memset(B, 0, sizeof(*B));
  Mem mem{al, (cudaStream_t)stream};
  Mem out{al, (cudaStream_t)stream};
  return with_output(B, out, [&] { return spref_impl(A, I, nI, J, nJ, B, mem, out, flags); });
}

int hs_sparse(const int32_t *i, const int32_t *j, const void *v, int64_t nnz, int64_t m, int64_t n, int dtype,
              int add_semiring, hs_mat *C, const hs_allocator *al, void *stream, uint32_t flags) {
  if (!C) return HS_EINVAL;
  memset(C, 0, sizeof(*C));
  Mem mem{al, (cudaStream_t)stream};
  Mem out{al, (cudaStream_t)stream};
  return with_output(C, out, [&] { return sparse_impl(i, j, v, nnz, m, n, dtype, add_semiring, C, mem, out, flags); });
}

int hs_spasgn(const hs_mat *A, const int32_t *I, int64_t nI, const int32_t *J, int64_t nJ, const hs_mat *B,
              int accumulate, int add_semiring, hs_mat *C, const hs_allocator *al, void *stream, uint32_t flags) {
  if (!C) return HS_EINVAL;
  memset(C, 0, sizeof(*C));
  Mem mem{al, (cudaStream_t)stream};
  Mem out{al, (cudaStream_t)stream};
  return with_output(C, out, [&] {
    return spasgn_impl(A, I, nI, J, nJ, B, accumulate, add_semiring, C, mem, out, flags);
  });
}

int hs_set_tuning(const hs_tuning *t) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune = t ? *t : k_tune_default;
  return HS_OK;
}

int hs_get_tuning(hs_tuning *t) {
  if (!t) return HS_EINVAL;
  std::lock_guard<std::mutex> g(g_tune_mu);
  *t = g_tune;
  return HS_OK;
}

void hs_mat_free(hs_mat *M, const hs_allocator *al, void *stream) {
  if (!M) return;
  Mem mem{al, (cudaStream_t)stream};
  free_mat(M, mem);
}

const char *hs_strerror(int s) {
  switch (s) {
    case HS_OK: return "success";
    case HS_EINVAL: return "invalid argument (shape, dtype, semiring, pointer or index)";
    case HS_ENONCANON: return "input matrix row not strictly increasing";
    case HS_EDUP: return "duplicate index in SpAsgn I or J";
    case HS_ENOMEM: return "allocation failed";
    case HS_ETIMEDOUT: return "bounded device wait expired";
    case HS_ECUDA: return "CUDA runtime error";
    case HS_EUNSUPPORTED: return "unsupported request";
    case HS_EINTERNAL: return "internal consistency check failed";
    case HS_ESCRATCH: return "product needs more scratch than the no-allocation entry point's fixed array";
    case HS_ECAPACITY: return "output capacity too small (C->nnz holds the size needed)";
  }
  return "unknown status";
}

int hs_last_cuda_error(void) { return t_last_cuda; }

const char *hs_last_error_detail(void) { return t_detail; }

int hs_version(void) { return 100; }

int64_t hs_launch_count(void) { return (int64_t)launch_total(); }

int hs_test_lookback_expiry(int spin_limit, int64_t withhold_tile) {
  if (spin_limit < 1 || withhold_tile < 0) return HS_EINVAL;
  t_sp_spin = spin_limit;
  t_sp_withhold = (long long)withhold_tile;
  return HS_OK;
}

void hs_profile_enable(int on) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.on = on != 0;
}

void hs_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.drain();
  for (auto &x : g_prof.ms) x = 0;
  for (auto &x : g_prof.launches) x = 0;
}

int hs_profile_read(double *ms, int64_t *launches, const char **names, int cap) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.drain();
  const int n = (int)g_prof.names.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (ms) ms[i] = g_prof.ms[i];
    if (launches) launches[i] = g_prof.launches[i];
    if (names) names[i] = g_prof.names[i].c_str();
  }
  return n;
}

}  // extern "C"
