// capi.cu -- the C ABI of libiluk (declared in include/iluk.h): handles,
// stream-ordered device memory, error reporting, the symbolic retry loop, the
// restarted GMRES(m) driver and the sweep-schedule autotuner.
//
// Host arithmetic (Givens rotations, back substitution of the small
// Hessenberg system) is compiled with FMA contraction off, one IEEE rounding
// per operation, like the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

using namespace iluk;

namespace {

int64_t initial_wait_limit() {
  // ILUK_WAIT_LIMIT_NS overrides the default bound on a single wait (20 s).
  const char *e = std::getenv("ILUK_WAIT_LIMIT_NS");
  if (e) {
    long long v = std::atoll(e);
    if (v > 0) return v;
  }
  return 20LL * 1000 * 1000 * 1000;
}
std::atomic<int64_t> g_wait_limit_ns{initial_wait_limit()};
std::atomic<int64_t> g_hold_row{-1};
std::atomic<int> g_sym_variant{0};
std::atomic<int64_t> g_launches{0};

struct DevCache {
  int sms = 0, smem = 0;
};
DevCache g_dev[64];
std::mutex g_dev_mu;

const DevCache &dev() {
  int d = 0;
  cudaGetDevice(&d);
  if (d < 0 || d >= 64) d = 0;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevCache &c = g_dev[d];
  if (c.sms == 0) {
    cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, d);
    cudaDeviceGetAttribute(&c.smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    if (c.sms <= 0) c.sms = 1;
    if (c.smem <= 0) c.smem = 48 * 1024;
    // The stream-ordered allocations (arenas, CSR arrays, Krylov vectors)
    // come from the device's default pool, which by default hands freed
    // memory back to the driver at every synchronisation, so each call maps
    // its hundreds of MB again.  Keep up to an eighth of the device's memory
    // (at most 16 GiB) cached in the pool instead; this process's pool only.
    cudaMemPool_t pool;
    size_t free_b = 0, total_b = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess &&
        cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      uint64_t keep = total_b / 8;
      if (keep > (16ull << 30)) keep = 16ull << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  return c;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMallocAsync((void **)p, count * sizeof(T), s);
}

template <typename T>
void dfree(T *&p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// Calls fn when the scope ends, whichever return leaves it, so that scratch
// buffers freed there with dfree do not leak when a CUDA call fails part-way
// (dfree nulls what it frees, so buffers freed earlier are skipped).
template <typename Fn>
struct ScopeExit {
  Fn fn;
  ~ScopeExit() { fn(); }
};
template <typename Fn>
ScopeExit<Fn> at_scope_exit(Fn fn) {
  return ScopeExit<Fn>{fn};
}

int fail(iluk_info *info, int st, int64_t row = -1, int64_t need = 0) {
  if (info) {
    info->status = st;
    info->row = row;
    info->need = need;
  }
  return st;
}

void info_init(iluk_info *info) {
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->row = -1;
  }
}

// Sizes and pointers of a pattern that the kernels may index: n and nnz not
// negative (n within int32 column indices), rowptr always present, colind
// present when nnz > 0.  Its contents are iluk_validate's business.
bool pattern_args_ok(const iluk_pattern *A) {
  return A && A->n >= 0 && A->n <= INT32_MAX && A->nnz >= 0 && A->rowptr &&
         (A->nnz == 0 || A->colind);
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return fail(info, _e == cudaErrorMemoryAllocation ? ILUK_ENOMEM : ILUK_ECUDA); \
  } while (0)

// Read a device error word; returns status and row.
int read_err(const DevErr *d, cudaStream_t s, int64_t *row, uint64_t *need) {
  DevErr h;
  cudaError_t e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ILUK_ECUDA;
  if (need) *need = h.need;
  if (h.key == kNoErr) {
    if (row) *row = -1;
    return ILUK_OK;
  }
  if (row) *row = (int64_t)(h.key >> 8);
  return (int)(h.key & 0xff);
}

int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

namespace iluk {
int64_t wait_limit() { return g_wait_limit_ns.load(); }
int64_t hold_row() { return g_hold_row.load(); }
int symbolic_variant() { return g_sym_variant.load(); }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
struct ProfRec {
  int kind;
  cudaEvent_t e0, e1;
};
std::atomic<bool> g_prof{false};
std::mutex g_prof_mu;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_on() { return g_prof.load(std::memory_order_relaxed); }

thread_local int prof_override = -1;

int prof_begin(int kind, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{kind, prof_event(), prof_event()};
  cudaEventRecord(r.e0, s);
  g_prof_recs.push_back(r);
  return (int)g_prof_recs.size() - 1;
}

void prof_end(int slot, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot >= 0 && slot < (int)g_prof_recs.size()) cudaEventRecord(g_prof_recs[slot].e1, s);
}
int num_sms() { return dev().sms; }
int max_smem_optin() { return dev().smem; }
}  // namespace iluk

extern "C" {

const char *iluk_strerror(int st) {
  switch (st) {
    case ILUK_OK: return "ok";
    case ILUK_EINVAL: return "invalid argument";
    case ILUK_EPATTERN: return "invalid CSR pattern";
    case ILUK_ENODIAG: return "missing diagonal entry";
    case ILUK_EZEROPIVOT: return "zero pivot";
    case ILUK_ENONFINITE: return "non-finite matrix value";
    case ILUK_ENOMEM: return "out of device memory or row too long";
    case ILUK_ETIMEOUT: return "bounded wait for another row gave up";
    case ILUK_ENOCONV: return "GMRES did not converge within maxit";
    case ILUK_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

int64_t iluk_set_wait_limit(int64_t ns) {
  if (ns <= 0) ns = 1;
  return g_wait_limit_ns.exchange(ns);
}

int64_t iluk_debug_hold_row(int64_t row) { return g_hold_row.exchange(row); }

int iluk_set_symbolic_variant(int variant) {
  if (variant < 0 || variant > 2) return -1;
  return g_sym_variant.exchange(variant);
}

int64_t iluk_launch_count(void) { return g_launches.load(); }

int iluk_prof_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (on) {
    for (auto &r : g_prof_recs) {
      cudaEventSynchronize(r.e1);
      g_prof_pool.push_back(r.e0);
      g_prof_pool.push_back(r.e1);
    }
    g_prof_recs.clear();
  }
  g_prof.store(on != 0);
  return ILUK_OK;
}

int iluk_prof_read(double *ms, int64_t *count, int nkinds) {
  if (nkinds < 0 || (nkinds > 0 && (!ms || !count))) return ILUK_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int k = 0; k < nkinds; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  for (auto &r : g_prof_recs) {
    if (r.kind < 0 || r.kind >= nkinds) continue;
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return ILUK_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) return ILUK_ECUDA;
    ms[r.kind] += t;
    count[r.kind] += 1;
  }
  return ILUK_OK;
}

int iluk_validate(const iluk_pattern *A, iluk_info *info, void *stream) {
  info_init(info);
  if (!pattern_args_ok(A)) return fail(info, ILUK_EINVAL);
  cudaStream_t s = (cudaStream_t)stream;
  DevErr *err = nullptr;
  auto scratch = at_scope_exit([&] { dfree(err, s); });
  CK(dalloc(&err, 1, s));
  CK(launch_fill_err(err, s));
  CK(launch_validate(A->n, A->nnz, A->rowptr, A->colind, err, s));
  int64_t row;
  int st = read_err(err, s, &row, nullptr);
  dfree(err, s);
  return fail(info, st, row);
}

void iluk_sym_destroy(iluk_sym *S) {
  if (!S) return;
  cudaStream_t s = 0;
  dfree(S->rowptr, s);
  dfree(S->colind, s);
  dfree(S->level, s);
  dfree(S->diag, s);
  dfree(S->arowptr, s);
  dfree(S->a2f, s);
  dfree(S->pinfo, s);
  dfree(S->tinfo, s);
  level_order_free(S->lord, s);
  level_order_free(S->uord, s);
  level_order_free(S->xlord, s);
  level_order_free(S->xuord, s);
  delete S;
}

int iluk_symbolic(const iluk_pattern *A, int k, iluk_sym **out, iluk_info *info, void *stream) {
  info_init(info);
  if (!out) return fail(info, ILUK_EINVAL);
  *out = nullptr;
  if (k < 0 || k > 250) return fail(info, ILUK_EINVAL);
  int st = iluk_validate(A, info, stream);
  if (st != ILUK_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n, nnz = A->nnz;

  iluk_sym *S = new iluk_sym();
  S->n = n;
  S->nnzA = nnz;
  S->k = k;
  DevErr *err = nullptr;
  SymArena ar{};
  int64_t *scan_tmp = nullptr;
  auto cleanup = [&]() {
    dfree(err, s);
    dfree(ar.col, s);
    dfree(ar.lev, s);
    dfree(ar.top, s);
    dfree(ar.row_off, s);
    dfree(ar.row_len, s);
    dfree(ar.row_ust, s);
    dfree(ar.meta, s);
    dfree(ar.ticket, s);
    dfree(scan_tmp, s);
  };
#define CKS(call)                                                   \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) {                                        \
      cleanup();                                                    \
      iluk_sym_destroy(S);                                          \
      return fail(info, _e == cudaErrorMemoryAllocation ? ILUK_ENOMEM : ILUK_ECUDA); \
    }                                                               \
  } while (0)

  CKS(dalloc(&err, 1, s));
  CKS(dalloc(&ar.row_off, n, s));
  CKS(dalloc(&ar.row_len, n, s));
  CKS(dalloc(&ar.row_ust, n, s));
  CKS(dalloc(&ar.meta, n, s));
  CKS(dalloc(&ar.ticket, 1, s));
  CKS(dalloc(&ar.top, 1, s));

  // Capacity of a row in shared memory and of the arena; grown on demand.
  int cap = k <= 1 ? 256 : 1024;
  int64_t mult = (k == 0) ? 1 : (k == 1) ? 8 : (k == 2) ? 17 : 65;
  int64_t arena_cap = nnz * mult + 1024;
  // level-map window of the symbolic walk (0: sorted lists only)
  int mapw = symbolic_map_width(n, A->rowptr, A->colind, k, s);
  if (symbolic_map_per_warp(mapw) + 5 * 1024 > (size_t)max_smem_optin()) mapw = 0;
  const int max_cap = (int)((max_smem_optin() - symbolic_map_per_warp(mapw)) / 5 / 32 * 32);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const int64_t arena_max = (int64_t)(free_b / 2 / 5);
  // room for the fill estimate plus what the per-warp chunks may leave unused
  int64_t floor_cap = -1, arena_floor = 0;
  auto floor_for_cap = [&]() {
    if (floor_cap != cap) {
      arena_floor = nnz * mult + 1024 + symbolic_arena_slack(n, k, cap, mapw, nnz * mult);
      floor_cap = cap;
    }
    return arena_floor;
  };
  arena_cap = floor_for_cap();
  if (arena_cap > arena_max) arena_cap = arena_max;

  for (int attempt = 0;; ++attempt) {
    if (ar.col && arena_cap < floor_for_cap() && floor_for_cap() <= arena_max) {  // cap grew
      dfree(ar.col, s);
      dfree(ar.lev, s);
      arena_cap = floor_for_cap();
    }
    if (!ar.col) {
      CKS(dalloc(&ar.col, arena_cap, s));
      CKS(dalloc(&ar.lev, arena_cap, s));
    }
    ar.cap = arena_cap;
    if (!symbolic_indep(k)) {  // rows wait on rows: announcements and arena start pending
      CKS(cudaMemsetAsync(ar.meta, 0xff, n * sizeof(unsigned long long), s));
      CKS(cudaMemsetAsync(ar.col, 0xff, arena_cap * sizeof(int32_t), s));
      CKS(cudaMemsetAsync(ar.lev, 0xff, arena_cap, s));
    }
    CKS(cudaMemsetAsync(ar.ticket, 0, sizeof(unsigned long long), s));
    CKS(cudaMemsetAsync(ar.top, 0, sizeof(unsigned long long), s));
    CKS(launch_fill_err(err, s));
    CKS(launch_symbolic_rows(n, A->rowptr, A->colind, k, ar, err, cap, mapw, s));
    int64_t row;
    uint64_t need = 0;
    st = read_err(err, s, &row, &need);
    if (st == ILUK_ECUDA) { cleanup(); iluk_sym_destroy(S); return fail(info, st); }
    if (st != ILUK_ENOMEM) {
      if (st != ILUK_OK) { cleanup(); iluk_sym_destroy(S); return fail(info, st, row); }
      break;
    }
    unsigned long long top = 0;
    CKS(cudaMemcpy(&top, ar.top, sizeof(top), cudaMemcpyDeviceToHost));
    if ((int64_t)need > cap) {
      if ((int64_t)need > max_cap) {
        cleanup(); iluk_sym_destroy(S);
        return fail(info, ILUK_ENOMEM, row, (int64_t)need);
      }
      cap = (int)next_pow2((int64_t)need);
      if (cap > max_cap) cap = max_cap;
    } else {
      int64_t want = arena_cap * 2;
      if ((int64_t)(top + top / 4) > want) want = (int64_t)(top + top / 4);
      if (want > arena_max) {
        cleanup(); iluk_sym_destroy(S);
        return fail(info, ILUK_ENOMEM, row, want * 5);
      }
      arena_cap = want;
      dfree(ar.col, s);
      dfree(ar.lev, s);
    }
    if (attempt > 40) { cleanup(); iluk_sym_destroy(S); return fail(info, ILUK_ENOMEM, row); }
  }

  // Compaction into CSR.
  CKS(dalloc(&S->rowptr, n + 1, s));
  CKS(dalloc(&scan_tmp, scan_tmp_elems(n), s));
  CKS(launch_scan_lengths(n, ar.row_len, S->rowptr, scan_tmp, s));
  int64_t nnzF = 0;
  CKS(cudaMemcpyAsync(&nnzF, S->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  S->nnz = nnzF;
  int32_t *maxrow = nullptr;
  CKS(dalloc(&S->colind, nnzF, s));
  CKS(dalloc(&S->level, nnzF, s));
  CKS(dalloc(&S->diag, n, s));
  CKS(dalloc(&S->a2f, nnz, s));
  CKS(dalloc(&S->arowptr, n + 1, s));
  CKS(dalloc(&maxrow, 1, s));
  CKS(cudaMemsetAsync(maxrow, 0, sizeof(int32_t), s));
  CKS(launch_symbolic_compact(n, ar, S->rowptr, S->colind, S->level, S->diag, maxrow, s));
  CKS(launch_a2f(n, A->rowptr, A->colind, S->rowptr, S->colind, S->a2f, s));
  CKS(dalloc(&S->pinfo, nnzF, s));
  CKS(launch_pivot_info(n, S->rowptr, S->colind, S->diag, S->pinfo, s));
  CKS(cudaMemcpyAsync(S->arowptr, A->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int32_t mr = 0;
  CKS(cudaMemcpyAsync(&mr, maxrow, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  S->max_row = mr;
  dfree(maxrow, s);
  cleanup();
  // The level orders of the two sweeps depend only on the pattern; they are
  // built by the first numeric phase, on a second stream while the
  // factorization runs (see ensure_levels).
#undef CKS
  *out = S;
  return fail(info, ILUK_OK);
}

// Build the sweeps' level orders of S once (synchronous on `s`).
static std::mutex g_levels_mu;
static int ensure_levels(const iluk_sym *Sc, cudaStream_t s) {
  iluk_sym *S = const_cast<iluk_sym *>(Sc);  // the level orders are a cache of the pattern
  std::lock_guard<std::mutex> lk(g_levels_mu);
  if (S->levels_built) return ILUK_OK;
  const int st = build_levels_pair(S->n, S->rowptr, S->colind, S->diag, &S->lord, &S->uord, s);
  if (st != ILUK_OK) return st;
  S->depth_lower = S->lord.nlev;
  S->depth_upper = S->uord.nlev;
  S->levels_built = true;
  return ILUK_OK;
}

int iluk_sym_query(const iluk_sym *S, iluk_sym_view *v) {
  if (!S || !v) return ILUK_EINVAL;
  v->n = S->n;
  v->nnz = S->nnz;
  v->rowptr = S->rowptr;
  v->colind = S->colind;
  v->level = S->level;
  v->diag = S->diag;
  v->a2f = S->a2f;
  v->max_row = S->max_row;
  v->depth_lower = S->depth_lower;
  v->depth_upper = S->depth_upper;
  v->k = S->k;
  return ILUK_OK;
}

int iluk_sym_export(const iluk_sym *S, int64_t *rowptr, int32_t *colind, uint8_t *level,
                    int64_t *diag, void *stream) {
  iluk_info *info = nullptr;
  if (!S) return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (rowptr) CK(cudaMemcpyAsync(rowptr, S->rowptr, (S->n + 1) * sizeof(int64_t), k, s));
  if (colind && S->nnz) CK(cudaMemcpyAsync(colind, S->colind, S->nnz * sizeof(int32_t), k, s));
  if (level && S->nnz) CK(cudaMemcpyAsync(level, S->level, S->nnz, k, s));
  if (diag && S->n) CK(cudaMemcpyAsync(diag, S->diag, S->n * sizeof(int64_t), k, s));
  return ILUK_OK;
}

int iluk_sym_depth(iluk_sym *S, int32_t *depth_lower, int32_t *depth_upper, void *stream) {
  if (!S) return ILUK_EINVAL;
  const int st = ensure_levels(S, (cudaStream_t)stream);
  if (st != ILUK_OK) return st;
  if (depth_lower) *depth_lower = S->depth_lower;
  if (depth_upper) *depth_upper = S->depth_upper;
  return ILUK_OK;
}

void iluk_fac_destroy(iluk_fac *F) {
  if (!F) return;
  cudaStream_t s = 0;
  dfree(F->val, s);
  dfree(F->sync, s);
  dfree(F->tmp, s);
  dfree(F->rdiag, s);
  dfree(F->err, s);
  dfree(F->trowptr, s);
  dfree(F->tcolind, s);
  dfree(F->tdiag, s);
  dfree(F->tval, s);
  level_order_free(F->tlord, s);
  level_order_free(F->tuord, s);
  dfree(F->aux.pre_s, s);
  dfree(F->aux.pre_k, s);
  dfree(F->aux.words, s);
  delete F;
}

static int numeric_into(iluk_fac *F, const double *A_val, iluk_info *info, cudaStream_t s,
                        bool build_levels = true, int32_t *depth = nullptr,
                        unsigned *maxdepth = nullptr) {
  const iluk_sym *S = F->S;
  // the numeric phase's row ticket lives in the handle's scratch
  CK(cudaMemsetAsync(F->sync, 0, sweep_sync_ints(S->n) * sizeof(int), s));
  CK(launch_fill_err(F->err, s));
  // the numeric phase also fills the reciprocals of the diagonal (after the factorization)
  CK(launch_numeric(S, A_val, F->val, F->rdiag, reinterpret_cast<unsigned long long *>(F->sync),
                    F->err, depth, maxdepth, s));
  // First factorization of this pattern: build the sweeps' level orders on a
  // second stream meanwhile (they read only the pattern; the numeric kernel
  // leaves room on every SM for the two level-building CTAs).
  int lst = ILUK_OK;
  if (build_levels && !S->levels_built) {
    cudaStream_t side = nullptr;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess) {
      prof_override = ILUK_PROF_OVERLAPPED;
      lst = ensure_levels(S, side);
      prof_override = -1;
      cudaStreamDestroy(side);
    } else {
      cudaGetLastError();
      lst = ensure_levels(S, s);
    }
  }
  int64_t row;
  int st = read_err(F->err, s, &row, nullptr);
  if (st == ILUK_OK && lst != ILUK_OK) st = lst;
  CK(launch_fill_err(F->err, s));
  // factor values changed: drop the transpose (its level orders depend only
  // on the pattern and are kept)
  dfree(F->trowptr, s);
  dfree(F->tcolind, s);
  dfree(F->tdiag, s);
  dfree(F->tval, s);
  return fail(info, st, row);
}

int iluk_numeric(const iluk_sym *S, const double *A_val, iluk_fac **out, iluk_info *info,
                 void *stream) {
  info_init(info);
  if (!S || !out || (!A_val && S->nnzA > 0)) return fail(info, ILUK_EINVAL);
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  iluk_fac *F = new iluk_fac();
  F->S = S;
  cudaError_t e = dalloc(&F->val, S->nnz, s);
  if (e == cudaSuccess) e = dalloc(&F->sync, sweep_sync_ints(S->n), s);
  if (e == cudaSuccess) e = dalloc(&F->tmp, S->n, s);
  if (e == cudaSuccess) e = dalloc(&F->rdiag, S->n, s);
  if (e == cudaSuccess) e = dalloc(&F->err, 2, s);
  if (e == cudaSuccess) e = launch_fill_pending(S->n, F->tmp, s);
  if (e != cudaSuccess) {
    iluk_fac_destroy(F);
    return fail(info, e == cudaErrorMemoryAllocation ? ILUK_ENOMEM : ILUK_ECUDA);
  }
  int st = numeric_into(F, A_val, info, s);
  if (st != ILUK_OK) {
    iluk_fac_destroy(F);
    return st;
  }
  *out = F;
  return ILUK_OK;
}

// iluk_symbolic + iluk_numeric with the two phases overlapped (k >= 2): one
// cooperative launch in which some CTAs walk the symbolic rows and the others
// factor each row as soon as its pattern is final (see k_factor_fused).  The
// results are those of the two calls bit for bit.  The sweeps of the returned
// factorization walk index orders until level orders are built (by a later
// iluk_numeric/iluk_refactor on S, or iluk_sym_depth).  Falls back to the two
// calls for k <= 1 (rows need no other rows' patterns) and whenever the fused
// launch cannot run or reports an error (the two calls then report it).
}  // extern "C"

// A factorization made without level orders (iluk_factor) measured the
// forward DAG's depth as it went: on a wide DAG the sweeps need level orders,
// so they are built now (on a narrow one index order is as fast).
static int levels_if_wide(const iluk_sym *S, const unsigned *maxdepth, iluk_info *info,
                          cudaStream_t s) {
  unsigned d = 0;
  CK(cudaMemcpyAsync(&d, maxdepth, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (d == 0 || S->n < kWideSweepRows * (int64_t)d) return ILUK_OK;
  return ensure_levels(S, s);
}

// iluk_factor, with two additions for iluk_solve: `validated` skips the
// pattern check the caller has made, and a non-null v0 asks the one-launch
// path to solve L x = v0 beside its numeric phase (each row's entry of x as
// soon as the row is factored).  Then *fwd_done tells whether it did: F->tmp
// holds x and must be consumed by a backward sweep before any other apply.
// The fallbacks (k <= 1, the two separate phases) leave *fwd_done false and
// F->tmp pending, as iluk_factor does.
static int factor_impl(const iluk_pattern *A, const double *A_val, int k, iluk_sym **S_out,
                       iluk_fac **F_out, iluk_info *info, void *stream, bool validated,
                       const double *v0, bool *fwd_done) {
  info_init(info);
  if (fwd_done) *fwd_done = false;
  if (!S_out || !F_out || !A || (!A_val && A->nnz > 0)) return fail(info, ILUK_EINVAL);
  *S_out = nullptr;
  *F_out = nullptr;
  if (k < 0 || k > 250) return fail(info, ILUK_EINVAL);
  auto two_phase = [&]() -> int {
    iluk_sym *S2 = nullptr;
    int st2 = iluk_symbolic(A, k, &S2, info, stream);
    if (st2 != ILUK_OK) return st2;
    iluk_fac *F2 = nullptr;
    st2 = iluk_numeric(S2, A_val, &F2, info, stream);
    if (st2 != ILUK_OK) {
      iluk_sym_destroy(S2);
      return st2;
    }
    *S_out = S2;
    *F_out = F2;
    return ILUK_OK;
  };
  // k <= 1: rows need no other rows' patterns, so the two phases simply run
  // one after the other, without the level orders (index orders instead)
  auto serial = [&]() -> int {
    cudaStream_t s2 = (cudaStream_t)stream;
    iluk_sym *S2 = nullptr;
    int st2 = iluk_symbolic(A, k, &S2, info, stream);
    if (st2 != ILUK_OK) return st2;
    iluk_fac *F2 = new iluk_fac();
    F2->S = S2;
    cudaError_t e2 = build_index_orders(S2->n, &S2->xlord, &S2->xuord, s2);
    if (e2 == cudaSuccess) e2 = dalloc(&F2->val, S2->nnz, s2);
    if (e2 == cudaSuccess) e2 = dalloc(&F2->sync, sweep_sync_ints(S2->n), s2);
    if (e2 == cudaSuccess) e2 = dalloc(&F2->tmp, S2->n, s2);
    if (e2 == cudaSuccess) e2 = dalloc(&F2->rdiag, S2->n, s2);
    if (e2 == cudaSuccess) e2 = dalloc(&F2->err, 2, s2);
    if (e2 == cudaSuccess) e2 = launch_fill_pending(S2->n, F2->tmp, s2);
    int32_t *depth = nullptr;
    unsigned *maxdepth = nullptr;
    auto depth_bufs = at_scope_exit([&] { dfree(depth, s2); dfree(maxdepth, s2); });
    if (e2 == cudaSuccess) e2 = dalloc(&depth, S2->n, s2);
    if (e2 == cudaSuccess) e2 = dalloc(&maxdepth, 1, s2);
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(depth, 0, (size_t)S2->n * sizeof(int32_t), s2);
    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(maxdepth, 0, sizeof(unsigned), s2);
    if (e2 != cudaSuccess) {
      iluk_fac_destroy(F2);
      iluk_sym_destroy(S2);
      return fail(info, e2 == cudaErrorMemoryAllocation ? ILUK_ENOMEM : ILUK_ECUDA);
    }
    st2 = numeric_into(F2, A_val, info, s2, false, depth, maxdepth);
    if (st2 == ILUK_OK) st2 = levels_if_wide(S2, maxdepth, info, s2);
    if (st2 != ILUK_OK) {
      iluk_fac_destroy(F2);
      iluk_sym_destroy(S2);
      return st2;
    }
    *S_out = S2;
    *F_out = F2;
    return ILUK_OK;
  };
  if (k <= 1 || A->n == 0) return serial();
  if (!validated) {
    int st = iluk_validate(A, info, stream);
    if (st != ILUK_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n, nnz = A->nnz;

  SymArena ar{};
  DevErr *err = nullptr;
  unsigned long long *rinfo = nullptr, *nticket = nullptr;
  double *aval_arena = nullptr;
  int64_t *scan_tmp = nullptr;
  int32_t *maxrow = nullptr;
  double *xf = nullptr;  // L^-1 v0, when asked for; becomes F->tmp
  DivPrep *rdiag = nullptr;  // the diagonal's reciprocals; becomes F->rdiag
  int32_t *fdepth = nullptr;  // each row's forward depth, and the DAG's
  unsigned *maxdepth = nullptr;
  iluk_sym *S = nullptr;
  iluk_fac *F = nullptr;
  auto cleanup = [&]() {
    dfree(xf, s);
    dfree(rdiag, s);
    dfree(fdepth, s);
    dfree(maxdepth, s);
    dfree(err, s);
    dfree(ar.col, s);
    dfree(ar.lev, s);
    dfree(ar.top, s);
    dfree(ar.row_off, s);
    dfree(ar.row_len, s);
    dfree(ar.row_ust, s);
    dfree(ar.meta, s);
    dfree(ar.ticket, s);
    dfree(rinfo, s);
    dfree(nticket, s);
    dfree(aval_arena, s);
    dfree(scan_tmp, s);
    dfree(maxrow, s);
  };
  // any failure of the fused path: the two separate phases instead
  auto fallback = [&]() -> int {
    cudaGetLastError();
    cleanup();
    if (F) iluk_fac_destroy(F);
    if (S) iluk_sym_destroy(S);
    F = nullptr;
    S = nullptr;
    return two_phase();
  };
#define CKF(call)                              \
  do {                                         \
    if ((call) != cudaSuccess) return fallback(); \
  } while (0)

  const int cap = 1024;  // symbolic row capacity, as iluk_symbolic starts with
  const int ncap = 512;  // numeric row capacity (longer rows of F: the two phases)
  const int64_t mult = k == 2 ? 17 : 65;
  int mapw = symbolic_map_width(n, A->rowptr, A->colind, k, s);
  if (symbolic_map_per_warp(mapw) + 5 * 1024 > (size_t)max_smem_optin()) mapw = 0;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  int64_t arena_cap = nnz * mult + 1024 + symbolic_arena_slack(n, k, cap, mapw, nnz * mult);
  if (arena_cap > (int64_t)(free_b / 2 / 13)) return fallback();  // 13 bytes an entry

  CKF(dalloc(&err, 1, s));
  CKF(dalloc(&ar.row_off, n, s));
  CKF(dalloc(&ar.row_len, n, s));
  CKF(dalloc(&ar.row_ust, n, s));
  CKF(dalloc(&ar.meta, n, s));
  CKF(dalloc(&ar.ticket, 1, s));
  CKF(dalloc(&ar.top, 1, s));
  CKF(dalloc(&ar.col, arena_cap, s));
  CKF(dalloc(&ar.lev, arena_cap, s));
  CKF(dalloc(&rinfo, n, s));
  CKF(dalloc(&nticket, 1, s));
  CKF(dalloc(&aval_arena, arena_cap, s));
  ar.cap = arena_cap;
  CKF(cudaMemsetAsync(ar.meta, 0xff, n * sizeof(unsigned long long), s));
  CKF(cudaMemsetAsync(rinfo, 0xff, n * sizeof(unsigned long long), s));
  CKF(cudaMemsetAsync(ar.col, 0xff, arena_cap * sizeof(int32_t), s));
  CKF(cudaMemsetAsync(ar.lev, 0xff, arena_cap, s));
  CKF(launch_fill_pending(arena_cap, aval_arena, s));
  CKF(cudaMemsetAsync(ar.ticket, 0, sizeof(unsigned long long), s));
  CKF(cudaMemsetAsync(nticket, 0, sizeof(unsigned long long), s));
  CKF(cudaMemsetAsync(ar.top, 0, sizeof(unsigned long long), s));
  CKF(launch_fill_err(err, s));
  if (v0) {
    CKF(dalloc(&xf, n, s));
    CKF(launch_fill_pending(n, xf, s));
  }
  CKF(dalloc(&rdiag, n, s));  // every row writes its own entry; ~0 marks the others
  CKF(cudaMemsetAsync(rdiag, 0xff, n * sizeof(DivPrep), s));
  CKF(dalloc(&fdepth, n, s));
  CKF(dalloc(&maxdepth, 1, s));
  CKF(cudaMemsetAsync(fdepth, 0, n * sizeof(int32_t), s));
  CKF(cudaMemsetAsync(maxdepth, 0, sizeof(unsigned), s));
  CKF(launch_factor_fused(n, nnz, A->rowptr, A->colind, A_val, k, ar, aval_arena, rinfo, nticket,
                          err, cap, mapw, ncap, v0, xf, rdiag, fdepth, maxdepth, s));
  {
    int64_t row = -1;
    uint64_t need = 0;
    if (read_err(err, s, &row, &need) != ILUK_OK) return fallback();
  }

  // the pattern into CSR, as iluk_symbolic does, and the values beside it
  S = new iluk_sym();
  S->n = n;
  S->nnzA = nnz;
  S->k = k;
  CKF(dalloc(&S->rowptr, n + 1, s));
  CKF(dalloc(&scan_tmp, scan_tmp_elems(n), s));
  CKF(launch_scan_lengths(n, ar.row_len, S->rowptr, scan_tmp, s));
  int64_t nnzF = 0;
  CKF(cudaMemcpyAsync(&nnzF, S->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  S->nnz = nnzF;
  CKF(dalloc(&S->colind, nnzF, s));
  CKF(dalloc(&S->level, nnzF, s));
  CKF(dalloc(&S->diag, n, s));
  CKF(dalloc(&S->a2f, nnz, s));
  CKF(dalloc(&S->arowptr, n + 1, s));
  CKF(dalloc(&maxrow, 1, s));
  CKF(cudaMemsetAsync(maxrow, 0, sizeof(int32_t), s));
  CKF(launch_symbolic_compact(n, ar, S->rowptr, S->colind, S->level, S->diag, maxrow, s));
  CKF(launch_a2f(n, A->rowptr, A->colind, S->rowptr, S->colind, S->a2f, s));
  CKF(dalloc(&S->pinfo, nnzF, s));
  CKF(launch_pivot_info(n, S->rowptr, S->colind, S->diag, S->pinfo, s));
  CKF(cudaMemcpyAsync(S->arowptr, A->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                      s));
  CKF(build_index_orders(n, &S->xlord, &S->xuord, s));
  F = new iluk_fac();
  F->S = S;
  CKF(dalloc(&F->val, nnzF, s));
  CKF(dalloc(&F->sync, sweep_sync_ints(n), s));
  if (xf) {
    F->tmp = xf;
    xf = nullptr;
  } else {
    CKF(dalloc(&F->tmp, n, s));
    CKF(launch_fill_pending(n, F->tmp, s));
  }
  F->rdiag = rdiag;  // written by the launch, row by row
  rdiag = nullptr;
  CKF(dalloc(&F->err, 2, s));
  CKF(launch_compact_values(n, ar, aval_arena, S->rowptr, F->val, s));
  CKF(launch_fill_err(F->err, s));
  int32_t mr = 0;
  CKF(cudaMemcpyAsync(&mr, maxrow, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CKF(cudaStreamSynchronize(s));
  S->max_row = mr;
  {
    iluk_info linfo;
    if (levels_if_wide(S, maxdepth, &linfo, s) != ILUK_OK) return fallback();
  }
#undef CKF
  cleanup();
  *S_out = S;
  *F_out = F;
  if (fwd_done) *fwd_done = v0 != nullptr;
  return fail(info, ILUK_OK);
}

extern "C" {

int iluk_factor(const iluk_pattern *A, const double *A_val, int k, iluk_sym **S_out,
                iluk_fac **F_out, iluk_info *info, void *stream) {
  return factor_impl(A, A_val, k, S_out, F_out, info, stream, false, nullptr, nullptr);
}

int iluk_refactor(iluk_fac *F, const double *A_val, iluk_info *info, void *stream) {
  info_init(info);
  if (!F || (!A_val && F->S->nnzA > 0)) return fail(info, ILUK_EINVAL);
  return numeric_into(F, A_val, info, (cudaStream_t)stream);
}

int iluk_fac_values(const iluk_fac *F, const double **val) {
  if (!F || !val) return ILUK_EINVAL;
  *val = F->val;
  return ILUK_OK;
}

int iluk_fac_export(const iluk_fac *F, double *val, void *stream) {
  iluk_info *info = nullptr;
  if (!F || !val) return ILUK_EINVAL;
  if (F->S->nnz)
    CK(cudaMemcpyAsync(val, F->val, F->S->nnz * sizeof(double), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
  return ILUK_OK;
}

int iluk_fac_status(iluk_fac *F, iluk_info *info, void *stream) {
  info_init(info);
  if (!F) return fail(info, ILUK_EINVAL);
  cudaStream_t s = (cudaStream_t)stream;
  int64_t row;
  int st = read_err(F->err, s, &row, nullptr);
  if (st != ILUK_OK) CK(launch_fill_pending(F->S->n, F->tmp, s));  // an aborted sweep
  CK(launch_fill_err(F->err, s));
  return fail(info, st, row);
}

static int ensure_transpose(iluk_fac *F, cudaStream_t s) {
  iluk_info *info = nullptr;
  if (F->trowptr) return ILUK_OK;
  const iluk_sym *S = F->S;
  int32_t *cursor = nullptr;
  int64_t *scan_tmp = nullptr;
  bool built = false;
  auto scratch = at_scope_exit([&] {
    dfree(cursor, s);
    dfree(scan_tmp, s);
    if (!built) {  // a failed build leaves no half-made transpose in F
      dfree(F->trowptr, s);
      dfree(F->tcolind, s);
      dfree(F->tdiag, s);
      dfree(F->tval, s);
    }
  });
  CK(dalloc(&F->trowptr, S->n + 1, s));
  CK(dalloc(&F->tcolind, S->nnz, s));
  CK(dalloc(&F->tdiag, S->n, s));
  CK(dalloc(&F->tval, S->nnz, s));
  CK(dalloc(&cursor, S->n, s));
  CK(dalloc(&scan_tmp, scan_tmp_elems(S->n), s));
  CK(launch_transpose(S->n, S->nnz, S->rowptr, S->colind, F->val, F->trowptr, F->tcolind,
                      F->tval, F->tdiag, cursor, scan_tmp, s));
  built = true;
  dfree(cursor, s);
  dfree(scan_tmp, s);
  if (!F->tlord.order && S->n) {
    int st = build_levels_pair(S->n, F->trowptr, F->tcolind, F->tdiag, &F->tlord, &F->tuord, s);
    if (st != ILUK_OK) return st;
  }
  return ILUK_OK;
}

// The helped sweeps' scratch (SweepAux), made the first time a schedule of F
// asks for ILUK_SCHED_WARP_CLUSTER_HELP; null while a stream capture runs
// (the helped kind then runs as WARP_CLUSTER) or if the memory is missing.
static const SweepAux *sweep_aux(iluk_fac *F, int sched, cudaStream_t s) {
  const bool want = (sched & 0xf) == ILUK_SCHED_WARP_CLUSTER_HELP ||
                    ((sched >> 8) & 0xf) == ILUK_SCHED_WARP_CLUSTER_HELP;
  if (!want) return nullptr;
  if (F->aux.pre_s) return &F->aux;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone) return nullptr;
  const int64_t n = F->S->n;
  SweepAux a;
  if (dalloc(&a.pre_s, n, s) != cudaSuccess || dalloc(&a.pre_k, n, s) != cudaSuccess ||
      dalloc(&a.words, 2, s) != cudaSuccess ||
      // no prefix carries epoch 0xffffffff, which the epochs never reach
      cudaMemsetAsync(a.pre_k, 0xff, (size_t)(n > 0 ? n : 1) * sizeof(unsigned long long), s) !=
          cudaSuccess ||
      cudaMemsetAsync(a.words, 0, 2 * sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    dfree(a.pre_s, s);
    dfree(a.pre_k, s);
    dfree(a.words, s);
    return nullptr;
  }
  a.n = n;
  F->aux = a;
  return &F->aux;
}

// Autotuner: time every sweep schedule (the warp-per-row ones at several CTA
// widths) on this factorization, forward and backward sweeps separately, and
// keep the fastest of each (packed as forward | backward << 8); the sweeps of
// the transpose (U^T then L^T, a different DAG) get their own pick, made the
// first time they run (the transpose must exist).  The sweeps' speed depends
// on the pattern, not on the values, so each pick is kept with the symbolic
// handle and a later factorization of the same pattern starts from it instead
// of timing again.  Skipped while the stream is being captured.
static int pick_schedule(iluk_fac *F, cudaStream_t s, bool transpose = false) {
  int &cur = transpose ? F->tsched : F->sched;
  int &hint = transpose ? F->S->tsched_hint : F->S->sched_hint;
  if (cur != ILUK_SCHED_AUTO) return cur;
  if (hint != ILUK_SCHED_AUTO) {
    cur = hint;
    return cur;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone) return ILUK_SCHED_WARP_GRID;
  const iluk_sym *S = F->S;
  // the trial sweeps use their own intermediate vector: F->tmp may hold a
  // forward sweep's result that a backward sweep has yet to consume
  double *p = nullptr, *y = nullptr, *t = nullptr;
  if (dalloc(&p, S->n, s) != cudaSuccess || dalloc(&y, S->n, s) != cudaSuccess ||
      dalloc(&t, S->n, s) != cudaSuccess) {
    dfree(p, s);
    dfree(y, s);
    return ILUK_SCHED_WARP_GRID;
  }
  // a right-hand side of ones: realistic operands for the divisions (zeros
  // would all take the IEEE fallback of the reciprocal division)
  launch_fill_value(S->n, p, 1.0, s);
  launch_fill_pending(S->n, t, s);
  float best_f = 1e30f, best_b = 1e30f;
  int pick_f = ILUK_SCHED_WARP_GRID, pick_b = ILUK_SCHED_WARP_GRID;
  const bool prof = g_prof.exchange(false);  // the trial runs are not profiled
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  // the warp-per-row kinds at several CTA widths: fewer warps keep fewer
  // rows in flight (less polling), more warps start each row earlier
  const int candidates[] = {ILUK_SCHED_FLAGS,
                            ILUK_SCHED_SINGLE_CTA,
                            ILUK_SCHED_CLUSTER,
                            ILUK_SCHED_WARP_GRID,
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_GRID, 512),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_GRID, 256),
                            ILUK_SCHED_WARP_CLUSTER,
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER, 768),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER, 512),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER, 384),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER, 256),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER_HELP, 512),
                            ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER_HELP, 384)};
  for (int sched : candidates) {
    float mf = 1e30f, mb = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      // the forward sweep alone, then the backward sweep alone, on the same
      // level orders the real applies use
      LevelOrder none;
      cudaEventRecord(e0, s);
      const SweepAux *aux = sweep_aux(F, sched, s);
      const cudaError_t ef =
          transpose ? launch_apply(S->n, F->trowptr, F->tcolind, F->tdiag, F->tval, F->rdiag,
                                   F->tlord, none, p, t, y, 1, sched, F->err, aux, s)
                    : launch_apply(S->n, S->rowptr, S->colind, S->diag, F->val, F->rdiag,
                                   sweep_fwd(S), none, p, t, y, 0, sched, F->err, aux, s);
      cudaEventRecord(e1, s);
      const cudaError_t eb =
          transpose ? launch_apply(S->n, F->trowptr, F->tcolind, F->tdiag, F->tval, F->rdiag,
                                   none, F->tuord, p, t, y, 1, sched, F->err, aux, s)
                    : launch_apply(S->n, S->rowptr, S->colind, S->diag, F->val, F->rdiag, none,
                                   sweep_bwd(S), p, t, y, 0, sched, F->err, aux, s);
      cudaEventRecord(e2, s);
      cudaEventSynchronize(e2);
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, e0, e1);
      cudaEventElapsedTime(&b, e1, e2);
      // a schedule this matrix cannot use (a launch that was refused) is not
      // a candidate
      if (ef != cudaSuccess) a = 1e30f;
      if (eb != cudaSuccess) b = 1e30f;
      if (ef != cudaSuccess || eb != cudaSuccess) cudaGetLastError();
      if (rep > 0) {
        if (a < mf) mf = a;
        if (b < mb) mb = b;
      }
    }
    if (mf < best_f) {
      best_f = mf;
      pick_f = sched;
    }
    if (mb < best_b) {
      best_b = mb;
      pick_b = sched;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  launch_fill_err(F->err, s);
  g_prof.store(prof);
  dfree(p, s);
  dfree(y, s);
  dfree(t, s);
  cur = pick_f | (pick_b << 8);
  hint = cur;
  return cur;
}

// The lockstep kinds (flags, single CTA, cluster) walk the padded level
// orders; a factorization from iluk_factor has only index orders until they
// are built, which happens here the first time such a schedule is used.
static int orders_for(iluk_fac *F, int sched, cudaStream_t s) {
  auto padded = [](int b) {
    const int kind = b & 0xf;
    return kind == ILUK_SCHED_FLAGS || kind == ILUK_SCHED_SINGLE_CTA ||
           kind == ILUK_SCHED_CLUSTER;
  };
  if (F->S->levels_built || !(padded(sched & 0xff) || padded((sched >> 8) & 0xff)))
    return ILUK_OK;
  return ensure_levels(F->S, s);
}

int iluk_apply_sched(iluk_fac *F, const double *p, double *y, int transpose, int sched,
                     void *stream) {
  iluk_info *info = nullptr;
  if (!F || (!p && F->S->n) || (!y && F->S->n)) return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const iluk_sym *S = F->S;
  if (transpose) {
    int st = ensure_transpose(F, s);
    if (st != ILUK_OK) return st;
  }
  if (sched == ILUK_SCHED_AUTO) sched = pick_schedule(F, s, transpose != 0);
  if (!transpose) {
    const int st = orders_for(F, sched, s);
    if (st != ILUK_OK) return st;
  }
  if (transpose) {
    CK(launch_apply(S->n, F->trowptr, F->tcolind, F->tdiag, F->tval, F->rdiag, F->tlord,
                    F->tuord, p, F->tmp, y, 1, sched, F->err, sweep_aux(F, sched, s), s));
  } else {
    CK(launch_apply(S->n, S->rowptr, S->colind, S->diag, F->val, F->rdiag, sweep_fwd(S),
                    sweep_bwd(S), p, F->tmp, y, 0, sched, F->err, sweep_aux(F, sched, s), s));
  }
  return ILUK_OK;
}

int iluk_apply(iluk_fac *F, const double *p, double *y, int transpose, void *stream) {
  return iluk_apply_sched(F, p, y, transpose, ILUK_SCHED_AUTO, stream);
}

}  // extern "C"

// A packed schedule (forward | backward << 8) that iluk_set_schedule takes:
// each byte a kind, plus a width (256..1024 threads) for the warp-per-row
// kinds only.
static bool sched_valid(int sched) {
  auto valid = [](int b) {
    const int kind = b & 0xf, w = (b >> 4) & 0xf;
    if (kind > ILUK_SCHED_WARP_CLUSTER_HELP) return false;
    return w == 0 || ((kind == ILUK_SCHED_WARP_GRID || kind == ILUK_SCHED_WARP_CLUSTER ||
                       kind == ILUK_SCHED_WARP_CLUSTER_HELP) &&
                      w >= 2 && w <= 8);
  };
  return sched >= 0 && sched <= 0xffff && valid(sched & 0xff) && valid((sched >> 8) & 0xff);
}

extern "C" {

int iluk_set_schedule(iluk_fac *F, int sched) {
  if (!F || !sched_valid(sched)) return ILUK_EINVAL;
  F->sched = sched;
  F->tsched = sched;
  return ILUK_OK;
}

int iluk_get_schedule(const iluk_fac *F) { return F ? F->sched : -1; }

void iiluk_destroy(iiluk *M) {
  if (!M) return;
  cudaStream_t s = 0;
  dfree(M->g, s);
  dfree(M->tmp, s);
  delete M;
}

int iiluk_build(const iluk_fac *F, iiluk **out, iluk_info *info, void *stream) {
  info_init(info);
  if (!F || !out) return fail(info, ILUK_EINVAL);
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const iluk_sym *S = F->S;
  iiluk *M = new iiluk();
  M->S = S;
  int *sync = nullptr;
  DevErr *err = nullptr;
  cudaError_t e = dalloc(&M->g, S->nnz, s);
  if (e == cudaSuccess) e = dalloc(&M->tmp, S->n, s);
  if (e == cudaSuccess) e = dalloc(&sync, 4, s);  // the build's row ticket
  if (e == cudaSuccess) e = dalloc(&err, 2, s);
  if (e == cudaSuccess) e = launch_fill_err(err, s);
  if (e == cudaSuccess) e = launch_fill_err(err + 1, s);
  if (e == cudaSuccess && !S->tinfo) {  // segment table, once per pattern
    iluk_sym *Sm = const_cast<iluk_sym *>(S);
    e = dalloc(&Sm->tinfo, S->nnz, s);
    if (e == cudaSuccess) e = launch_tpiilu_info(S->n, S->rowptr, S->colind, S->diag, Sm->tinfo, s);
  }
  if (e == cudaSuccess) e = launch_iiluk_build(S, F->val, F->rdiag, S->tinfo, M->g, sync, err, s);
  int st = ILUK_OK;
  int64_t row = -1;
  if (e == cudaSuccess) {
    int64_t r0, r1;
    int s0 = read_err(err, s, &r0, nullptr);
    int s1 = read_err(err + 1, s, &r1, nullptr);
    if (s0 != ILUK_OK) { st = s0; row = r0; }
    else if (s1 != ILUK_OK) { st = s1; row = S->n - 1 - r1; }
  } else {
    st = e == cudaErrorMemoryAllocation ? ILUK_ENOMEM : ILUK_ECUDA;
  }
  dfree(sync, s);
  dfree(err, s);
  if (st != ILUK_OK) {
    iiluk_destroy(M);
    return fail(info, st, row);
  }
  *out = M;
  return fail(info, ILUK_OK);
}

int iiluk_values(const iiluk *M, const double **g) {
  if (!M || !g) return ILUK_EINVAL;
  *g = M->g;
  return ILUK_OK;
}

int iiluk_export(const iiluk *M, double *g, void *stream) {
  iluk_info *info = nullptr;
  if (!M || !g) return ILUK_EINVAL;
  if (M->S->nnz)
    CK(cudaMemcpyAsync(g, M->g, M->S->nnz * sizeof(double), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
  return ILUK_OK;
}

int iiluk_apply(const iiluk *M, const double *p, double *y, void *stream) {
  iluk_info *info = nullptr;
  if (!M || (M->S->n > 0 && (!p || !y))) return ILUK_EINVAL;
  CK(launch_iiluk_apply(M->S, M->g, p, M->tmp, y, (cudaStream_t)stream));
  return ILUK_OK;
}

int iluk_spmv(const iluk_pattern *A, const double *A_val, const double *x, double *y,
              void *stream) {
  iluk_info *info = nullptr;
  if (!pattern_args_ok(A) || (A->n > 0 && (!x || !y)) || (A->nnz > 0 && !A_val))
    return ILUK_EINVAL;
  CK(launch_spmv(A->n, A->rowptr, A->colind, A_val, x, y, nullptr, (cudaStream_t)stream));
  return ILUK_OK;
}

int iluk_div_rn(int64_t n, const double *a, const double *b, double *q, void *stream) {
  iluk_info *info = nullptr;
  if (n < 0 || (n > 0 && (!a || !b || !q))) return ILUK_EINVAL;
  CK(launch_div_check(n, a, b, q, (cudaStream_t)stream));
  return ILUK_OK;
}

int iluk_dot(int64_t n, const double *x, const double *y, double *out, void *stream) {
  iluk_info *info = nullptr;
  if (n < 0 || !out || (n > 0 && (!x || !y))) return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DotScratch ds{};
  auto scratch = at_scope_exit([&] {
    dfree(ds.partial, s);
    dfree(ds.counter, s);
  });
  CK(dalloc(&ds.partial, kDotP, s));
  CK(dalloc(&ds.counter, 1, s));
  CK(cudaMemsetAsync(ds.counter, 0, sizeof(unsigned), s));
  CK(launch_dot(n, x, y, out, 0, ds, s));
  dfree(ds.partial, s);
  dfree(ds.counter, s);
  return ILUK_OK;
}

int iluk_transpose(const iluk_pattern *A, const double *A_val, int64_t *t_rowptr,
                   int32_t *t_colind, double *t_val, void *stream) {
  iluk_info *info = nullptr;
  if (!pattern_args_ok(A) || !t_rowptr || (A->nnz > 0 && (!A_val || !t_colind || !t_val)))
    return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *cursor = nullptr;
  int64_t *scan_tmp = nullptr;
  auto scratch = at_scope_exit([&] { dfree(cursor, s); dfree(scan_tmp, s); });
  if (A->n > 0) {
    CK(dalloc(&cursor, A->n, s));
    CK(dalloc(&scan_tmp, scan_tmp_elems(A->n), s));
  }
  CK(launch_transpose(A->n, A->nnz, A->rowptr, A->colind, A_val, t_rowptr, t_colind, t_val,
                      nullptr, cursor, scan_tmp, s));
  return ILUK_OK;
}

int iluk_adjoint_scatter(const iluk_pattern *A, const double *lambda, const double *x, double *gA,
                         void *stream) {
  iluk_info *info = nullptr;
  if (!pattern_args_ok(A) || (A->n > 0 && (!lambda || !x)) || (A->nnz > 0 && !gA))
    return ILUK_EINVAL;
  CK(launch_adjoint_scatter(A->n, A->rowptr, A->colind, lambda, x, gA, (cudaStream_t)stream));
  return ILUK_OK;
}

int iluk_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *A_vals, double *F_vals,
                         iluk_info *infos, void *stream) {
  iluk_info *info = nullptr;
  if (!S || nbatch < 0) return ILUK_EINVAL;
  if (nbatch == 0) return ILUK_OK;
  if ((S->nnzA > 0 && !A_vals) || (S->nnz > 0 && !F_vals)) return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *ticket = nullptr;
  DevErr *errs = nullptr;
  auto scratch = at_scope_exit([&] {
    dfree(ticket, s);
    dfree(errs, s);
  });
  CK(dalloc(&ticket, 1, s));
  CK(dalloc(&errs, nbatch, s));
  CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(errs, 0xff, nbatch * sizeof(DevErr), s));
  CK(launch_numeric_batched(S, nbatch, A_vals, F_vals, ticket, errs, s));
  std::vector<DevErr> h(nbatch);
  CK(cudaMemcpyAsync(h.data(), errs, nbatch * sizeof(DevErr), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  dfree(ticket, s);
  dfree(errs, s);
  int first = ILUK_OK;
  for (int64_t b = 0; b < nbatch; ++b) {
    int st = h[b].key == kNoErr ? ILUK_OK : (int)(h[b].key & 0xff);
    if (infos) {
      std::memset(&infos[b], 0, sizeof(iluk_info));
      infos[b].status = st;
      infos[b].row = st == ILUK_OK ? -1 : (int64_t)(h[b].key >> 8);
    }
    if (first == ILUK_OK && st != ILUK_OK) first = st;
  }
  return first;
}

// ---------------------------------------------------------------------------
// Batched persistent solve
// ---------------------------------------------------------------------------
}  // extern "C"

struct iluk_batch {
  int64_t nitems = 0;
  int restart = 30, maxit = 10000, cap = 32, width = 0;
  bool spin = false;  // in-CTA sweeps polling values instead of level barriers
  double rtol = 1e-8;
  int64_t nwork = 0;  // work slots (CTAs of the widest grid)
  std::vector<int64_t> order;  // ticket t runs item order[t]: largest items first
  void *items = nullptr, *results = nullptr, *work = nullptr;
  unsigned long long *ticket = nullptr;
  std::vector<double *> bufs;
};

extern "C" {

void iluk_batch_destroy(iluk_batch *B) {
  if (!B) return;
  cudaStream_t s = 0;
  for (auto p : B->bufs) cudaFreeAsync(p, s);
  if (B->items) cudaFreeAsync(B->items, s);
  if (B->results) cudaFreeAsync(B->results, s);
  if (B->work) cudaFreeAsync(B->work, s);
  if (B->ticket) cudaFreeAsync(B->ticket, s);
  delete B;
}

int iluk_batch_create(const iluk_batch_item *items, int64_t nitems, int restart, double rtol,
                      int maxit, iluk_batch **out, void *stream) {
  iluk_info *info = nullptr;
  if (!out || nitems < 0 || (nitems > 0 && !items) || restart < 1 ||
      restart > batch_max_restart() || maxit < 0)
    return ILUK_EINVAL;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  iluk_batch *B = new iluk_batch();
  B->nitems = nitems;
  B->restart = restart;
  B->rtol = rtol;
  B->maxit = maxit;
  int64_t maxn = 1, maxf = 1;
  int maxrow = 1;
  std::vector<unsigned char> hitems(batch_item_bytes() * (nitems ? nitems : 1));
  for (int64_t i = 0; i < nitems; ++i) {
    const iluk_batch_item &it = items[i];
    if (!it.S || !it.a_rowptr || !it.b || !it.x || (it.S->nnzA && (!it.a_colind || !it.a_val))) {
      delete B;
      return ILUK_EINVAL;
    }
  }
  // The CTAs take items in ticket order.  Handing out the largest first
  // (longest-processing-time list scheduling) keeps a large item from
  // starting last and running on alone; an item's cost is its FP64 work per
  // iteration, the entries of F and A plus a few vectors.
  B->order.resize(nitems);
  std::vector<int64_t> cost(nitems);
  for (int64_t i = 0; i < nitems; ++i) {
    B->order[i] = i;
    cost[i] = items[i].S->nnz + items[i].S->nnzA + 4 * items[i].S->n;
  }
  std::stable_sort(B->order.begin(), B->order.end(),
                   [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  for (int64_t t = 0; t < nitems; ++t) {
    const iluk_batch_item &it = items[B->order[t]];
    const int lst = ensure_levels(it.S, s);  // the in-CTA sweeps walk the level orders
    if (lst != ILUK_OK) {
      delete B;
      return lst;
    }
    batch_pack_item(hitems.data() + t * batch_item_bytes(), it.S, it.a_rowptr, it.a_colind,
                    it.a_val, it.b, it.x);
    if (it.S->n > maxn) maxn = it.S->n;
    if (it.S->nnz > maxf) maxf = it.S->nnz;
    if (it.S->max_row > maxrow) maxrow = it.S->max_row;
  }
  B->cap = (maxrow + 31) & ~31;
  if (batch_smem_bytes(1024, B->cap, restart) + 8 * 1024 > (size_t)max_smem_optin()) {
    delete B;
    return ILUK_ENOMEM;  // a row of F too long for the per-warp slices
  }
  // Work slots: enough for the widest grid (up to four 256-thread CTAs per
  // SM), and no more than there are items.
  B->nwork = 4 * (int64_t)num_sms();
  if (B->nwork > nitems) B->nwork = nitems > 0 ? nitems : 1;
  const int64_t ldv = maxn;
  auto cleanup = [&]() { iluk_batch_destroy(B); };
  if (dalloc((unsigned char **)&B->items, hitems.size(), s) != cudaSuccess ||
      dalloc((unsigned char **)&B->results, batch_result_bytes() * (nitems ? nitems : 1), s) !=
          cudaSuccess ||
      dalloc((unsigned char **)&B->work, batch_work_bytes() * B->nwork, s) != cudaSuccess ||
      dalloc(&B->ticket, 1, s) != cudaSuccess) {
    cleanup();
    return ILUK_ENOMEM;
  }
  std::vector<unsigned char> hwork(batch_work_bytes() * B->nwork);
  for (int64_t w = 0; w < B->nwork; ++w) {
    double *fval, *V, *vw, *z, *u, *tmp;
    if (dalloc(&fval, maxf, s) != cudaSuccess || (B->bufs.push_back(fval), false) ||
        dalloc(&V, (size_t)ldv * (restart + 1), s) != cudaSuccess ||
        (B->bufs.push_back(V), false) || dalloc(&vw, ldv, s) != cudaSuccess ||
        (B->bufs.push_back(vw), false) || dalloc(&z, (size_t)ldv * restart, s) != cudaSuccess ||
        (B->bufs.push_back(z), false) || dalloc(&u, ldv, s) != cudaSuccess ||
        (B->bufs.push_back(u), false) || dalloc(&tmp, ldv, s) != cudaSuccess) {
      cleanup();
      return ILUK_ENOMEM;
    }
    B->bufs.push_back(tmp);
    batch_pack_work(hwork.data() + w * batch_work_bytes(), fval, V, vw, z, u, tmp, ldv);
  }
  CK(cudaMemcpyAsync(B->items, hitems.data(), hitems.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(B->work, hwork.data(), hwork.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  *out = B;
  return ILUK_OK;
}

static cudaError_t batch_launch(iluk_batch *B, int width, bool spin, cudaStream_t s) {
  return launch_batch_solve(width, spin, B->items, B->nitems, B->results, B->work, B->nwork,
                            B->ticket, B->restart, B->rtol, B->maxit, B->cap, s);
}

int iluk_batch_solve(iluk_batch *B, void *stream) {
  iluk_info *info = nullptr;
  if (!B) return ILUK_EINVAL;
  if (B->nitems == 0) return ILUK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (B->width == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      B->width = 1024;
    } else {
      // Autotuner: run the whole batch at each width, with level-barrier
      // sweeps and with spinning sweeps, and keep the fastest.
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      for (bool sp : {false, true})
        for (int w : {256, 512, 1024}) {
          cudaEventRecord(e0, s);
          CK(batch_launch(B, w, sp, s));
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) {
            best = ms;
            B->width = w;
            B->spin = sp;
          }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      // results do not depend on the width or the schedule: the last run holds them
      return ILUK_OK;
    }
  }
  CK(batch_launch(B, B->width, B->spin, s));
  return ILUK_OK;
}

int iluk_batch_width(const iluk_batch *B) { return B ? B->width : 0; }

int iluk_batch_spin(const iluk_batch *B) { return B && B->spin ? 1 : 0; }

int iluk_batch_set_schedule(iluk_batch *B, int width, int spin) {
  if (!B || (width != 256 && width != 512 && width != 1024)) return ILUK_EINVAL;
  B->width = width;
  B->spin = spin != 0;
  return ILUK_OK;
}

int iluk_batch_results(iluk_batch *B, iluk_info *infos, void *stream) {
  iluk_info *info = nullptr;
  if (!B) return ILUK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<unsigned char> h(batch_result_bytes() * (B->nitems ? B->nitems : 1));
  CK(cudaMemcpyAsync(h.data(), B->results, batch_result_bytes() * B->nitems,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int first = ILUK_OK;
  std::vector<int64_t> slot(B->nitems);  // result slot of each item
  for (int64_t t = 0; t < B->nitems; ++t) slot[B->order[t]] = t;
  for (int64_t i = 0; i < B->nitems; ++i) {
    int32_t st, it, cyc;
    int64_t row;
    double rel;
    batch_unpack_result(h.data() + slot[i] * batch_result_bytes(), &st, &it, &cyc, &row, &rel);
    if (infos) {
      std::memset(&infos[i], 0, sizeof(iluk_info));
      infos[i].status = st;
      infos[i].iters = it;
      infos[i].cycles = cyc;
      infos[i].row = row;
      infos[i].relres = rel;
    }
    if (first == ILUK_OK && st != ILUK_OK) first = st;
  }
  return first;
}

// ---------------------------------------------------------------------------
// GMRES(m)
// ---------------------------------------------------------------------------
int gmres_solve(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                const double *b, double *x, int m, double rtol, int maxit, int transpose,
                iluk_info *info, void *stream) {
  return gmres_solve_ex(A, A_val, prec_kind, prec, b, x, m, rtol, maxit, transpose,
                        ILUK_BASIS_AUTO, info, stream);
}

}  // extern "C"

// The ILU(k) factorization made inside GMRES once v_1 = r_0 / ||r_0|| is
// known (iluk_solve): it may solve L x = v_1 beside its numeric phase, which
// saves the first application its forward sweep.  Returns an iluk status;
// on success *F is the factorization and *fwd_done whether F->tmp holds
// L^-1 v_1; on failure finfo describes it.
struct FactorHook {
  virtual int operator()(const double *v1, iluk_fac **F, bool *fwd_done, iluk_info *finfo) = 0;
  virtual ~FactorHook() = default;
};

static int gmres_impl(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                      const double *b, double *x, int m, double rtol, int maxit, int transpose,
                      int basis, iluk_info *info, void *stream, FactorHook *hook) {
  info_init(info);
  if (!pattern_args_ok(A) || m < 1 || maxit < 0) return fail(info, ILUK_EINVAL);
  if (basis < ILUK_BASIS_AUTO || basis > ILUK_BASIS_MINV_VY) return fail(info, ILUK_EINVAL);
  if ((A->n > 0 && (!b || !x)) || (A->nnz > 0 && !A_val)) return fail(info, ILUK_EINVAL);
  if (prec_kind != ILUK_PREC_NONE && !prec && !hook) return fail(info, ILUK_EINVAL);
  if (transpose && prec_kind == ILUK_PREC_IILU) return fail(info, ILUK_EINVAL);
  if (hook && (transpose || prec_kind != ILUK_PREC_ILU)) return fail(info, ILUK_EINVAL);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n;
  iluk_fac *F = prec_kind == ILUK_PREC_ILU ? (iluk_fac *)prec : nullptr;
  iiluk *M = prec_kind == ILUK_PREC_IILU ? (iiluk *)prec : nullptr;

  // operator rows: A, or the explicit transpose of A
  const int64_t *orp = A->rowptr;
  const int32_t *oci = A->colind;
  const double *ov = A_val;
  int64_t *trp = nullptr;
  int32_t *tci = nullptr;
  double *tv = nullptr;
  int32_t *cursor = nullptr;
  int64_t *scan_tmp = nullptr;
  // With ILUK_BASIS_STORE, Z keeps the preconditioned basis z_j = M^-1 v_j
  // of a cycle, which ends with x += Z y (the flexible-GMRES form: no extra
  // application of M).  Without it only V is kept: RECOMPUTE applies M to
  // each v_j again at the end of the cycle and accumulates Z y in the same
  // order (the same bits, m more applications), MINV_VY forms x += M^-1 (V y).
  double *V = nullptr, *Z = nullptr, *w = nullptr, *u = nullptr, *Hd = nullptr, *dsc = nullptr,
         *dy = nullptr;
  DotScratch ds{};
  auto scratch = at_scope_exit([&] {
    dfree(cursor, s); dfree(scan_tmp, s); dfree(trp, s); dfree(tci, s); dfree(tv, s);
    dfree(V, s); dfree(Z, s); dfree(w, s); dfree(u, s); dfree(Hd, s); dfree(dsc, s);
    dfree(dy, s); dfree(ds.partial, s); dfree(ds.counter, s);
  });
  if (transpose) {
    CK(dalloc(&trp, n + 1, s));
    CK(dalloc(&tci, A->nnz, s));
    CK(dalloc(&tv, A->nnz, s));
    CK(dalloc(&cursor, n, s));
    CK(dalloc(&scan_tmp, scan_tmp_elems(n), s));
    CK(launch_transpose(n, A->nnz, A->rowptr, A->colind, A_val, trp, tci, tv, nullptr, cursor,
                        scan_tmp, s));
    dfree(cursor, s);
    dfree(scan_tmp, s);
    orp = trp;
    oci = tci;
    ov = tv;
  }
  const int64_t ldv = n > 0 ? n : 1;
  if (basis == ILUK_BASIS_AUTO) {
    // keep Z only when its m vectors take at most half of the free memory
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double need = (double)ldv * (double)m * sizeof(double);
    basis = need <= 0.5 * (double)free_b ? ILUK_BASIS_STORE : ILUK_BASIS_RECOMPUTE;
  }
  const bool store_z = basis == ILUK_BASIS_STORE;
  CK(dalloc(&V, (size_t)ldv * (m + 1), s));
  CK(dalloc(&Z, store_z ? (size_t)ldv * m : (size_t)ldv, s));
  CK(dalloc(&w, ldv, s));
  CK(dalloc(&u, ldv, s));
  CK(dalloc(&Hd, (size_t)(m + 1) * m, s));
  CK(dalloc(&dsc, 4, s));
  CK(dalloc(&dy, m, s));
  CK(dalloc(&ds.partial, kDotP, s));
  CK(dalloc(&ds.counter, 1, s));
  CK(cudaMemsetAsync(ds.counter, 0, sizeof(unsigned), s));
  if (F && transpose) {
    int st = ensure_transpose(F, s);
    if (st != ILUK_OK) return fail(info, st);
  }
  int sched = F ? pick_schedule(F, s, transpose != 0) : 0;
  if (F && !transpose) {
    const int st = orders_for(F, sched, s);
    if (st != ILUK_OK) return fail(info, st);
  }
  bool fwd_ready = false;  // F->tmp holds L^-1 v_1 (made by the factorization)
  // an exit before the backward sweep consumed it leaves F->tmp armed again,
  // as every later application expects
  auto rearm = at_scope_exit([&] {
    if (fwd_ready && F) launch_fill_pending(n, F->tmp, s);
  });

  auto precond = [&](const double *in, double *outv) -> cudaError_t {
    if (F) {
      if (transpose)
        return launch_apply(n, F->trowptr, F->tcolind, F->tdiag, F->tval, F->rdiag, F->tlord,
                            F->tuord, in, F->tmp, outv, 1, sched, F->err, sweep_aux(F, sched, s),
                            s);
      return launch_apply(n, F->S->rowptr, F->S->colind, F->S->diag, F->val, F->rdiag,
                          sweep_fwd(F->S), sweep_bwd(F->S), in, F->tmp, outv, 0, sched, F->err,
                          sweep_aux(F, sched, s), s);
    }
    if (M) return launch_iiluk_apply(M->S, M->g, in, M->tmp, outv, s);
    return cudaMemcpyAsync(outv, in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  };

  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gv(m + 1), yv(m),
      col(m + 2);
  int status = ILUK_ENOCONV;
  int iters = 0, cycles = 0;
  double relres = 0.0;
  double bnorm = 0.0;
  CK(launch_dot(n, b, b, dsc + 0, 1, ds, s));
  CK(cudaMemcpyAsync(&bnorm, dsc + 0, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  if (bnorm == 0.0) {
    status = ILUK_OK;
  } else {
    for (;;) {
      // r = b - A x  (r lives in w)
      CK(launch_spmv(n, orp, oci, ov, x, w, b, s));
      CK(launch_dot(n, w, w, dsc + 1, 1, ds, s));
      double beta = 0.0;
      CK(cudaMemcpyAsync(&beta, dsc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      relres = beta / bnorm;
      if (relres <= rtol) { status = ILUK_OK; break; }
      if (iters >= maxit) { status = ILUK_ENOCONV; break; }
      ++cycles;
      CK(launch_scale_div(n, w, dsc + 1, V, s));
      if (hook && !F) {
        iluk_info finfo;
        const int hst = (*hook)(V, &F, &fwd_ready, &finfo);
        if (hst != ILUK_OK) {
          if (info) *info = finfo;
          return hst;
        }
        sched = pick_schedule(F, s);
        const int ost = orders_for(F, sched, s);
        if (ost != ILUK_OK) return fail(info, ost);
      }
      gv[0] = beta;
      int jend = -1;
      bool bad = false;
      for (int j = 0; j < m; ++j) {
        double *vj = V + (size_t)j * ldv;
        double *hc = Hd + (size_t)j * (m + 1);  // column j of H
        double *zj = store_z ? Z + (size_t)j * ldv : Z;
        if (fwd_ready) {  // z_1 from the forward sweep the factorization made
          fwd_ready = false;
          CK(launch_apply_backward(n, F->S->rowptr, F->S->colind, F->S->diag, F->val, F->rdiag,
                                   sweep_bwd(F->S), F->tmp, zj, sched, F->err,
                                   sweep_aux(F, sched, s), s));
        } else {
          CK(precond(vj, zj));
        }
        CK(launch_spmv(n, orp, oci, ov, zj, w, nullptr, s));
        CK(launch_dot(n, w, V, hc + 0, 0, ds, s));
        for (int i = 0; i <= j; ++i) {
          const double *vi = V + (size_t)i * ldv;
          if (i < j)
            CK(launch_mgs_step(n, w, vi, hc + i, V + (size_t)(i + 1) * ldv, hc + i + 1, 0, ds, s));
          else
            CK(launch_mgs_step(n, w, vi, hc + i, w, hc + j + 1, 1, ds, s));
        }
        CK(launch_scale_div(n, w, hc + j + 1, V + (size_t)(j + 1) * ldv, s));
        CK(cudaMemcpyAsync(col.data(), hc, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = col[i];
        const double hn = col[j + 1];
        for (int i = 0; i < j; ++i) {  // previous rotations
          const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
          const double t1 = cs[i] * a, t2 = sn[i] * c;
          const double t3 = sn[i] * a, t4 = cs[i] * c;
          H[(size_t)i * m + j] = t1 + t2;
          H[(size_t)(i + 1) * m + j] = t4 - t3;
        }
        const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
        const double aa = a * a, cc = c * c;
        const double rr = std::sqrt(aa + cc);
        if (rr == 0.0) { bad = true; break; }
        cs[j] = a / rr;
        sn[j] = c / rr;
        H[(size_t)j * m + j] = rr;
        H[(size_t)(j + 1) * m + j] = 0.0;
        gv[j + 1] = -(sn[j] * gv[j]);
        gv[j] = cs[j] * gv[j];
        ++iters;
        jend = j;
        const bool breakdown = hn == 0.0;
        if (std::fabs(gv[j + 1]) / bnorm <= rtol || iters >= maxit || breakdown) break;
      }
      if (bad) { status = ILUK_EINVAL; break; }
      for (int i = jend; i >= 0; --i) {
        double sacc = gv[i];
        for (int l = i + 1; l <= jend; ++l) {
          const double prod = H[(size_t)i * m + l] * yv[l];
          sacc = sacc - prod;
        }
        yv[i] = sacc / H[(size_t)i * m + i];
      }
      CK(cudaMemcpyAsync(dy, yv.data(), (jend + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
      if (store_z) {
        CK(launch_combine(n, Z, ldv, dy, jend + 1, u, s));
        CK(launch_add(n, x, u, s));
      } else if (basis == ILUK_BASIS_RECOMPUTE) {
        // u = sum_j y_j z_j from +0.0, one term at a time, z_j recomputed
        CK(cudaMemsetAsync(u, 0, n * sizeof(double), s));
        for (int j = 0; j <= jend; ++j) {
          CK(precond(V + (size_t)j * ldv, Z));
          CK(launch_acc_scaled(n, u, dy + j, Z, s));
        }
        CK(launch_add(n, x, u, s));
      } else {  // ILUK_BASIS_MINV_VY
        CK(launch_combine(n, V, ldv, dy, jend + 1, u, s));
        CK(precond(u, Z));
        CK(launch_add(n, x, Z, s));
      }
    }
  }
  CK(cudaStreamSynchronize(s));
  int64_t prow = -1;
  if (F) {
    int pst = read_err(F->err, s, &prow, nullptr);
    if (pst != ILUK_OK) {
      launch_fill_err(F->err, s);
      launch_fill_pending(n, F->tmp, s);
      status = pst;
    }
  }
  dfree(V, s); dfree(Z, s); dfree(w, s); dfree(u, s); dfree(Hd, s); dfree(dsc, s); dfree(dy, s);
  dfree(ds.partial, s); dfree(ds.counter, s);
  dfree(trp, s); dfree(tci, s); dfree(tv, s);
  if (info) {
    info->status = status;
    info->iters = iters;
    info->relres = relres;
    info->cycles = cycles;
    info->row = prow;
  }
  return status;
}

extern "C" {

int gmres_solve_ex(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                   const double *b, double *x, int m, double rtol, int maxit, int transpose,
                   int basis, iluk_info *info, void *stream) {
  return gmres_impl(A, A_val, prec_kind, prec, b, x, m, rtol, maxit, transpose, basis, info,
                    stream, nullptr);
}

int iluk_solve(const iluk_pattern *A, const double *A_val, int k, const double *b, double *x,
               int m, double rtol, int maxit, int sched, iluk_sym **S_out, iluk_fac **F_out,
               iluk_info *info, void *stream) {
  info_init(info);
  if (S_out) *S_out = nullptr;
  if (F_out) *F_out = nullptr;
  if (!pattern_args_ok(A) || (A->nnz > 0 && !A_val) || (A->n > 0 && (!b || !x)) || k < 0 ||
      k > 250 || m < 1 || maxit < 0 || !sched_valid(sched))
    return fail(info, ILUK_EINVAL);
  int st = iluk_validate(A, info, stream);
  if (st != ILUK_OK) return st;
  struct Hook : FactorHook {
    const iluk_pattern *A;
    const double *A_val;
    int k, sched;
    void *stream;
    iluk_sym *S = nullptr;
    iluk_fac *F = nullptr;
    int operator()(const double *v1, iluk_fac **Fo, bool *fwd_done, iluk_info *finfo) override {
      int st2 = factor_impl(A, A_val, k, &S, &F, finfo, stream, true, v1, fwd_done);
      if (st2 == ILUK_OK) st2 = iluk_set_schedule(F, sched);
      if (st2 != ILUK_OK) {
        if (F) iluk_fac_destroy(F);
        if (S) iluk_sym_destroy(S);
        F = nullptr;
        S = nullptr;
        *fwd_done = false;
        return st2;
      }
      *Fo = F;
      return ILUK_OK;
    }
  } hook;
  hook.A = A;
  hook.A_val = A_val;
  hook.k = k;
  hook.sched = sched;
  hook.stream = stream;
  st = gmres_impl(A, A_val, ILUK_PREC_ILU, nullptr, b, x, m, rtol, maxit, 0, ILUK_BASIS_AUTO,
                  info, stream, &hook);
  if (!hook.F && st == ILUK_OK) {
    // GMRES ended before its first application (b = 0, or x = 0 already
    // within rtol): the factorization still runs, and its failures count
    iluk_info finfo;
    const int fst = factor_impl(A, A_val, k, &hook.S, &hook.F, &finfo, stream, true, nullptr,
                                nullptr);
    if (fst != ILUK_OK) {
      if (info) *info = finfo;
      return fst;
    }
    iluk_set_schedule(hook.F, sched);
  }
  if (F_out && S_out && hook.F) {
    *S_out = hook.S;
    *F_out = hook.F;
  } else {
    if (hook.F) iluk_fac_destroy(hook.F);
    if (hook.S) iluk_sym_destroy(hook.S);
  }
  return st;
}

int bicgstab_solve(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                   const double *b, double *x, double rtol, int maxit, iluk_info *info,
                   void *stream) {
  info_init(info);
  if (!pattern_args_ok(A) || maxit < 0) return fail(info, ILUK_EINVAL);
  if ((A->n > 0 && (!b || !x)) || (A->nnz > 0 && !A_val)) return fail(info, ILUK_EINVAL);
  if (prec_kind != ILUK_PREC_NONE && !prec) return fail(info, ILUK_EINVAL);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n;
  iluk_fac *F = prec_kind == ILUK_PREC_ILU ? (iluk_fac *)prec : nullptr;
  iiluk *M = prec_kind == ILUK_PREC_IILU ? (iiluk *)prec : nullptr;
  const int64_t ld = n > 0 ? n : 1;
  double *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *ph = nullptr, *sv = nullptr,
         *sh = nullptr, *t = nullptr, *dsc = nullptr;
  DotScratch ds{};
  auto scratch = at_scope_exit([&] {
    dfree(r, s); dfree(rh, s); dfree(p, s); dfree(v, s); dfree(ph, s); dfree(sv, s);
    dfree(sh, s); dfree(t, s); dfree(dsc, s); dfree(ds.partial, s); dfree(ds.counter, s);
  });
  CK(dalloc(&r, ld, s));
  CK(dalloc(&rh, ld, s));
  CK(dalloc(&p, ld, s));
  CK(dalloc(&v, ld, s));
  CK(dalloc(&ph, ld, s));
  CK(dalloc(&sv, ld, s));
  CK(dalloc(&sh, ld, s));
  CK(dalloc(&t, ld, s));
  CK(dalloc(&dsc, 8, s));
  CK(dalloc(&ds.partial, kDotP, s));
  CK(dalloc(&ds.counter, 1, s));
  CK(cudaMemsetAsync(ds.counter, 0, sizeof(unsigned), s));
  const int sched = F ? pick_schedule(F, s) : 0;
  if (F) {
    const int st = orders_for(F, sched, s);
    if (st != ILUK_OK) return fail(info, st);
  }
  auto precond = [&](const double *in, double *outv) -> cudaError_t {
    if (F)
      return launch_apply(n, F->S->rowptr, F->S->colind, F->S->diag, F->val, F->rdiag,
                          sweep_fwd(F->S), sweep_bwd(F->S), in, F->tmp, outv, 0, sched, F->err,
                          sweep_aux(F, sched, s), s);
    if (M) return launch_iiluk_apply(M->S, M->g, in, M->tmp, outv, s);
    return cudaMemcpyAsync(outv, in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  };
  // scalars come back to the host, as in gmres_solve: dsc[0..k) per sync
  double hs[4] = {0.0, 0.0, 0.0, 0.0};
  auto fetch = [&](int cnt) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hs, dsc, cnt * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  };
  int status = ILUK_ENOCONV, iters = 0;
  double relres = 0.0;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  CK(launch_dot(n, b, b, dsc, 1, ds, s));
  CK(fetch(1));
  const double bnorm = hs[0];
  if (bnorm == 0.0) {
    status = ILUK_OK;
  } else {
    CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(rh, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(launch_dot(n, rh, r, dsc, 0, ds, s));
    CK(fetch(1));
    double rho = hs[0], rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    for (int it = 1; it <= maxit; ++it) {
      if (rho == 0.0) { status = ILUK_EINVAL; break; }
      if (it == 1) {
        CK(cudaMemcpyAsync(p, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      } else {
        const double b1 = rho / rho_prev, b2 = alpha / omega;
        CK(launch_bicg_dir(n, p, r, v, b1 * b2, omega, s));
      }
      CK(precond(p, ph));
      CK(launch_spmv(n, A->rowptr, A->colind, A_val, ph, v, nullptr, s));
      CK(launch_dot(n, rh, v, dsc, 0, ds, s));
      CK(fetch(1));
      const double sigma = hs[0];
      if (sigma == 0.0) { status = ILUK_EINVAL; break; }
      alpha = rho / sigma;
      CK(launch_axmy(n, sv, r, alpha, v, s));
      CK(launch_dot(n, sv, sv, dsc, 1, ds, s));
      CK(fetch(1));
      iters = it;
      if (hs[0] / bnorm <= rtol) {  // converged at the half step
        CK(launch_bicg_x(n, x, alpha, ph, 0.0, nullptr, s));
        status = ILUK_OK;
        break;
      }
      CK(precond(sv, sh));
      CK(launch_spmv(n, A->rowptr, A->colind, A_val, sh, t, nullptr, s));
      CK(launch_dot(n, t, t, dsc, 0, ds, s));
      CK(launch_dot(n, t, sv, dsc + 1, 0, ds, s));
      CK(fetch(2));
      const double tt = hs[0], ts = hs[1];
      if (tt == 0.0) { status = ILUK_EINVAL; break; }
      omega = ts / tt;
      CK(launch_bicg_x(n, x, alpha, ph, omega, sh, s));
      CK(launch_axmy(n, r, sv, omega, t, s));
      CK(launch_dot(n, r, r, dsc, 1, ds, s));
      CK(launch_dot(n, rh, r, dsc + 1, 0, ds, s));  // the next rho, fetched together
      CK(fetch(2));
      if (hs[0] / bnorm <= rtol) { status = ILUK_OK; break; }
      if (omega == 0.0) { status = ILUK_EINVAL; break; }
      rho_prev = rho;
      rho = hs[1];
    }
    // the true residual ||b - A x|| / ||b||
    CK(launch_spmv(n, A->rowptr, A->colind, A_val, x, t, b, s));
    CK(launch_dot(n, t, t, dsc, 1, ds, s));
    CK(fetch(1));
    relres = hs[0] / bnorm;
  }
  CK(cudaStreamSynchronize(s));
  int64_t prow = -1;
  if (F) {
    int pst = read_err(F->err, s, &prow, nullptr);
    if (pst != ILUK_OK) {
      launch_fill_err(F->err, s);
      launch_fill_pending(n, F->tmp, s);
      status = pst;
    }
  }
  dfree(r, s); dfree(rh, s); dfree(p, s); dfree(v, s); dfree(ph, s); dfree(sv, s); dfree(sh, s);
  dfree(t, s); dfree(dsc, s); dfree(ds.partial, s); dfree(ds.counter, s);
  if (info) {
    info->status = status;
    info->iters = iters;
    info->relres = relres;
    info->cycles = 0;
    info->row = prow;
  }
  return status;
}

// One solve from host buffers: the arrays cross to the device and x comes
// back inside the call, around the same device calls a caller would make
// (pattern check, symbolic + numeric, GMRES with the ILU(k) sweeps).
int iluk_solve_host(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                    const double *val, const double *b, double *x, int k, int restart,
                    double rtol, int maxit, int sched, iluk_info *info, void *stream) {
  info_init(info);
  if (n < 0 || nnz < 0 || !rowptr || (nnz > 0 && (!colind || !val)) || (n > 0 && (!b || !x)) ||
      k < 0 || k > 250 || restart < 1 || maxit < 0)
    return fail(info, ILUK_EINVAL);
  cudaStream_t s = (cudaStream_t)stream;
  int64_t *d_rp = nullptr;
  int32_t *d_ci = nullptr;
  double *d_v = nullptr, *d_b = nullptr, *d_x = nullptr;
  iluk_sym *S = nullptr;
  iluk_fac *F = nullptr;
  auto scratch = at_scope_exit([&] {
    if (F) iluk_fac_destroy(F);
    if (S) iluk_sym_destroy(S);
    dfree(d_rp, s); dfree(d_ci, s); dfree(d_v, s); dfree(d_b, s); dfree(d_x, s);
  });
  const size_t nn = n > 0 ? (size_t)n : 1, nz = nnz > 0 ? (size_t)nnz : 1;
  CK(dalloc(&d_rp, (size_t)n + 1, s));
  CK(dalloc(&d_ci, nz, s));
  CK(dalloc(&d_v, nz, s));
  CK(dalloc(&d_b, nn, s));
  CK(dalloc(&d_x, nn, s));
  CK(cudaMemcpyAsync(d_rp, rowptr, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (nnz > 0) {
    CK(cudaMemcpyAsync(d_ci, colind, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_v, val, (size_t)nnz * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (n > 0) CK(cudaMemcpyAsync(d_b, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
  const iluk_pattern A{n, nnz, d_rp, d_ci};
  const int st = iluk_solve(&A, d_v, k, d_b, d_x, restart, rtol, maxit, sched, nullptr, nullptr,
                            info, stream);
  if (st != ILUK_OK && st != ILUK_ENOCONV) return st;
  if (n > 0) CK(cudaMemcpyAsync(x, d_x, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

int tpilu_solve(const iluk_pattern *A, const double *A_val, iluk_fac *F, iiluk *M, int solver,
                const double *b, double *x, int m, double rtol, int iilu_maxit, int maxit,
                int *used, iluk_info *info, void *stream) {
  info_init(info);
  if (!pattern_args_ok(A) || !F || !used ||
      (solver != ILUK_SOLVER_GMRES && solver != ILUK_SOLVER_BICGSTAB) || iilu_maxit < 0 ||
      maxit < 0 || (solver == ILUK_SOLVER_GMRES && m < 1))
    return fail(info, ILUK_EINVAL);
  if ((A->n > 0 && (!b || !x)) || (A->nnz > 0 && !A_val)) return fail(info, ILUK_EINVAL);
  auto run = [&](int kind, void *prec, int its) {
    return solver == ILUK_SOLVER_GMRES
               ? gmres_solve(A, A_val, kind, prec, b, x, m, rtol, its, 0, info, stream)
               : bicgstab_solve(A, A_val, kind, prec, b, x, rtol, its, info, stream);
  };
  iiluk *own = nullptr;
  if (!M) {
    const int bst = iiluk_build(F, &own, info, stream);
    if (bst != ILUK_OK) return bst;
    M = own;
  }
  int st = run(ILUK_PREC_IILU, M, iilu_maxit);
  iiluk_destroy(own);
  *used = ILUK_PREC_IILU;
  // a failed sweep status (time-out) is not a convergence failure: report it
  if (st == ILUK_OK || (st != ILUK_ENOCONV && st != ILUK_EINVAL)) return st;
  *used = ILUK_PREC_ILU;
  return run(ILUK_PREC_ILU, F, maxit);
}

}  // extern "C"
