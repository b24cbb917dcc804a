// internal.h -- host-side declarations shared by the libiluk translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

// Rows of one sweep DAG in level order, every level padded with -1 to a
// multiple of 32 entries (see levels.cu).
// Where the cluster warp-per-row sweep keeps x_i: in the shared memory of the
// CTA that computes row i (rank << 26 | slot), which depends on the order,
// the cluster width and the CTA width; built on first use.
struct OwnerCode {
  int C = 0, threads = 0;
  int32_t *code = nullptr;
};

struct LevelOrder {
  int32_t *order = nullptr;   // levels padded to multiples of 32 slots (-1 fills)
  int64_t *lstart = nullptr;  // int64[nlev+1]: first slot of each level
  int64_t len = 0;
  int32_t nlev = 0;
  int32_t *corder = nullptr;  // the same rows without padding (clen = rows)
  int64_t clen = 0;
  OwnerCode owner[8];         // cache, see OwnerCode
};
void level_order_free(LevelOrder &lo, cudaStream_t s);

// Handle layouts (opaque in the public header).
struct iluk_sym {
  int64_t n = 0, nnz = 0, nnzA = 0;
  int k = 0;
  int64_t *rowptr = nullptr;   // F pattern
  int32_t *colind = nullptr;
  uint8_t *level = nullptr;
  int64_t *diag = nullptr;
  int64_t *arowptr = nullptr;  // copy of A's row pointers
  int32_t *a2f = nullptr;      // offset of each A entry inside its F row
  int64_t *pinfo = nullptr;    // per lower entry (i,h): diag position of row h << 24 | |U(h)|
  int64_t *tinfo = nullptr;    // per entry (i,h): row h's TPIILU segment (start << 24 | length),
                               // built by the first iiluk_build on the pattern
  int32_t max_row = 0;
  int32_t depth_lower = -1, depth_upper = -1;
  LevelOrder lord, uord;       // forward / backward sweep level orders
  bool levels_built = false;   // lord/uord are built by the first numeric phase
  LevelOrder xlord, xuord;     // index orders (iluk_factor), for the sweeps until lord/uord exist
  // the sweep schedules the autotuner picked for a factorization of this
  // pattern, for the sweeps of F and of its transpose (0: none yet); later
  // factorizations of the pattern start from them
  mutable int sched_hint = 0, tsched_hint = 0;
};

// The orders the sweeps of S walk: the level orders once built, else the
// index orders of a factorization that skipped them.
inline const LevelOrder &sweep_fwd(const iluk_sym *S) { return S->levels_built ? S->lord : S->xlord; }
inline const LevelOrder &sweep_bwd(const iluk_sym *S) { return S->levels_built ? S->uord : S->xuord; }

namespace iluk {
// Scratch of the helped warp-per-row sweeps (ILUK_SCHED_WARP_CLUSTER_HELP):
// per row the prefix a helper published (the partial difference, and the
// launch's epoch << 32 | the number of entries it covers), then two words:
// the current epoch (starts at 1) and the count of CTAs of the running launch
// that have finished.
struct SweepAux {
  double *pre_s = nullptr;
  unsigned long long *pre_k = nullptr;
  unsigned *words = nullptr;
  int64_t n = 0;
};
}  // namespace iluk

struct iluk_fac {
  const iluk_sym *S = nullptr;
  double *val = nullptr;          // F values
  int *sync = nullptr;            // tickets + flags for sweeps: see sweeps.cu
  double *tmp = nullptr;          // intermediate vector of the two sweeps
  iluk::DivPrep *rdiag = nullptr; // the diagonal with its fixed-point reciprocals (from
                                  // the numeric phase; used by every sweep division)
  iluk::DevErr *err = nullptr;    // status of asynchronous calls
  // explicit transpose of F for (L~U~)^-T, built on first use
  int64_t *trowptr = nullptr;
  int32_t *tcolind = nullptr;
  int64_t *tdiag = nullptr;
  double *tval = nullptr;
  LevelOrder tlord, tuord;        // level orders of the transposed sweeps
  int sched = 0;                  // schedule picked for the sweeps (ILUK_SCHED_*)
  int tsched = 0;                 // and for the transposed sweeps
  iluk::SweepAux aux;             // helped sweeps' scratch, made on first use
};

struct iiluk {
  const iluk_sym *S = nullptr;
  double *g = nullptr;
  double *tmp = nullptr;
};

namespace iluk {

// Average rows per forward level from which the row kernels (numeric phase,
// TPIILU build) walking level order leave out the column map for more warps.
constexpr int64_t kWideLevelRows = 300;
// Average rows per forward level from which a factorization made without
// level orders builds them for its sweeps: on DAGs this wide the sweeps in
// index order starve (C3, 378 rows a level: one application 8.7 ms in index
// order, 1.5 ms in level order; 27-point 90^3, 1,168 a level: 22.1 / 2.2 ms),
// on narrower ones index order is as fast or faster (2D 256^2, 64 a level:
// 1.06 / 1.35 ms; the random band, 10 a level: 15.1 / 15.3 ms).
constexpr int64_t kWideSweepRows = 128;

int64_t wait_limit();
void note_launch();              // counts kernel launches (iluk_launch_count)

// Optional per-kernel timing with CUDA events on the launching stream
// (iluk_prof_enable / iluk_prof_read).  Kinds are listed in include/iluk.h.
bool prof_on();
int prof_begin(int kind, cudaStream_t s);
// While >= 0, every scope opened by this thread is counted under this kind.
extern thread_local int prof_override;
void prof_end(int slot, cudaStream_t s);
struct ProfScope {
  int slot;
  cudaStream_t s;
  ProfScope(int kind, cudaStream_t st)
      : slot(prof_on() ? prof_begin(prof_override >= 0 ? prof_override : kind, st) : -1),
        s(st) {}
  ~ProfScope() {
    if (slot >= 0) prof_end(slot, s);
  }
};
int64_t hold_row();
// The symbolic walk for k <= 1 (iluk_set_symbolic_variant): 0 independent
// rows in ascending order, 1 independent rows in descending order, 2 the
// general walk with waits (as for k >= 2).
int symbolic_variant();
inline bool symbolic_indep(int k) { return k <= 1 && symbolic_variant() != 2; }              // test hook: a row whose flag is never published

// Sizes of the persistent grids (filled on first use per device).
int num_sms();
int max_smem_optin();

// Validation / utilities (validate.cu)
cudaError_t launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                            DevErr *err, cudaStream_t s);
// out[0] = 0, out[i+1] = sum_{r<=i} len[r]  (int32 lengths -> int64 offsets)
cudaError_t launch_scan_lengths(int64_t n, const int32_t *len, int64_t *out, int64_t *tmp,
                                cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_fill_err(DevErr *err, cudaStream_t s);

// Symbolic (symbolic.cu)
struct SymArena {
  int32_t *col; uint8_t *lev; int64_t cap; unsigned long long *top;
  int64_t *row_off; int32_t *row_len; int32_t *row_ust;
  unsigned long long *meta; unsigned long long *ticket;
};
cudaError_t launch_symbolic_rows(int64_t n, const int64_t *arp, const int32_t *aci, int k,
                                 const SymArena &ar, DevErr *err, int cap, int mapw,
                                 cudaStream_t s);
int symbolic_map_width(int64_t n, const int64_t *arp, const int32_t *aci, int k, cudaStream_t s);
size_t symbolic_smem_per_warp(int cap);
size_t symbolic_map_per_warp(int mapw);  // per-warp shared memory of the level map
// arena entries the per-warp chunks may leave unused, for this shape
int64_t symbolic_arena_slack(int64_t n, int k, int cap, int mapw, int64_t rows_est);
int64_t symbolic_chunk(int k, int cap);
cudaError_t launch_compact_values(int64_t n, const SymArena &ar, const double *aval,
                                  const int64_t *frp, double *fval, cudaStream_t s);
cudaError_t launch_factor_fused(int64_t n, int64_t nnz_a, const int64_t *arp,
                                const int32_t *aci, const double *aval, int k, const SymArena &ar,
                                double *arena_val, unsigned long long *rinfo,
                                unsigned long long *num_ticket, DevErr *err, int scap, int mapw,
                                int ncap, const double *v0, double *xf, DivPrep *rdiag,
                                int32_t *depth, unsigned *maxdepth, cudaStream_t s);
cudaError_t build_index_orders(int64_t n, LevelOrder *fwd, LevelOrder *bwd, cudaStream_t s);
cudaError_t launch_symbolic_compact(int64_t n, const SymArena &ar, const int64_t *frp,
                                    int32_t *fci, uint8_t *flev, int64_t *fdiag, int32_t *maxrow,
                                    cudaStream_t s);
cudaError_t launch_a2f(int64_t n, const int64_t *arp, const int32_t *aci, const int64_t *frp,
                       const int32_t *fci, int32_t *a2f, cudaStream_t s);

// Levels (levels.cu): synchronous; allocates both orders on success.
int build_levels_pair(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                      LevelOrder *fwd, LevelOrder *bwd, cudaStream_t s);

// Numeric (numeric.cu)
// The factor values double as ready flags (numeric.cu); fval is overwritten.
cudaError_t launch_pivot_info(int64_t n, const int64_t *frp, const int32_t *fci,
                              const int64_t *fdiag, int64_t *pinfo, cudaStream_t s);
// depth/maxdepth (may be null): each row's forward depth and the DAG's
// depth, zeroed by the caller.
cudaError_t launch_numeric(const iluk_sym *S, const double *aval, double *fval, DivPrep *rdiag,
                           unsigned long long *ticket, DevErr *err, int32_t *depth,
                           unsigned *maxdepth, cudaStream_t s);
cudaError_t launch_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *avals,
                                   double *fvals, unsigned long long *ticket, DevErr *errs,
                                   cudaStream_t s);

// Sweeps (sweeps.cu)
size_t sweep_sync_ints(int64_t n);
// The backward half of launch_apply alone, for a tmp that already holds
// L^-1 p (the factorization computed it beside the numeric phase).
cudaError_t launch_apply_backward(int64_t n, const int64_t *rp, const int32_t *ci,
                                  const int64_t *dg, const double *v, const DivPrep *rd,
                                  const LevelOrder &bwd, double *tmp, double *y, int sched,
                                  DevErr *err, const SweepAux *aux, cudaStream_t s);
// y = (LU)^-1 p (or ^-T on the transposed arrays).  tmp must hold the pending
// marker in every entry on entry, and does again on exit.
cudaError_t launch_apply(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                         const double *v, const DivPrep *rd, const LevelOrder &fwd,
                         const LevelOrder &bwd,
                         const double *p, double *tmp, double *y, int transpose, int sched,
                         DevErr *err, const SweepAux *aux, cudaStream_t s);
cudaError_t launch_fill_pending(int64_t n, double *x, cudaStream_t s);
cudaError_t launch_fill_value(int64_t n, double *x, double v, cudaStream_t s);
cudaError_t launch_div_check(int64_t n, const double *a, const double *b, double *q,
                             cudaStream_t s);
cudaError_t launch_transpose(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                             const double *v, int64_t *trp, int32_t *tci, double *tv,
                             int64_t *tdiag, int32_t *cursor, int64_t *scan_tmp, cudaStream_t s);

// TPIILU (tpiilu.cu)
cudaError_t launch_iiluk_build(const iluk_sym *S, const double *fval, const DivPrep *rdiag,
                               const int64_t *tinfo, double *g, int *sync, DevErr *err,
                               cudaStream_t s);
cudaError_t launch_tpiilu_info(int64_t n, const int64_t *frp, const int32_t *fci,
                               const int64_t *fdiag, int64_t *tinfo, cudaStream_t s);
cudaError_t launch_iiluk_apply(const iluk_sym *S, const double *g, const double *p, double *tmp,
                               double *y, cudaStream_t s);

// Krylov pieces (krylov.cu)
constexpr int kDotP = 4096;
struct DotScratch { double *partial; unsigned int *counter; };
cudaError_t launch_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        const double *x, double *y, const double *b_minus, cudaStream_t s);
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *out, int take_sqrt,
                       const DotScratch &ds, cudaStream_t s);
cudaError_t launch_mgs_step(int64_t n, double *w, const double *vi, const double *hij,
                            const double *vnext, double *out, int take_sqrt,
                            const DotScratch &ds, cudaStream_t s);
cudaError_t launch_scale_div(int64_t n, const double *x, const double *den, double *y,
                             cudaStream_t s);
cudaError_t launch_combine(int64_t n, const double *V, int64_t ldv, const double *y, int cnt,
                           double *u, cudaStream_t s);
cudaError_t launch_add(int64_t n, double *x, const double *z, cudaStream_t s);
cudaError_t launch_acc_scaled(int64_t n, double *u, const double *y, const double *z,
                              cudaStream_t s);
cudaError_t launch_bicg_dir(int64_t n, double *p, const double *r, const double *v, double beta,
                            double omega, cudaStream_t s);
cudaError_t launch_axmy(int64_t n, double *out, const double *a, double alpha, const double *b,
                        cudaStream_t s);
cudaError_t launch_bicg_x(int64_t n, double *x, double alpha, const double *ph, double omega,
                          const double *sh, cudaStream_t s);
cudaError_t launch_adjoint_scatter(int64_t n, const int64_t *rp, const int32_t *ci,
                                   const double *lam, const double *x, double *gA,
                                   cudaStream_t s);

// Batched persistent solve (batched.cu)
size_t batch_item_bytes();
size_t batch_result_bytes();
size_t batch_work_bytes();
size_t batch_smem_bytes(int nt, int cap, int m);
int batch_max_restart();
void batch_pack_item(void *dst, const iluk_sym *S, const int64_t *arp, const int32_t *aci,
                     const double *aval, const double *b, double *x);
void batch_pack_work(void *dst, double *fval, double *V, double *w, double *z, double *u,
                     double *tmp, int64_t ldv);
void batch_unpack_result(const void *src, int32_t *status, int32_t *iters, int32_t *cycles,
                         int64_t *row, double *relres);
cudaError_t launch_batch_solve(int nt, bool spin, const void *items, int64_t nitems,
                               void *results, void *work, int64_t nwork,
                               unsigned long long *ticket, int m, double rtol, int maxit, int cap,
                               cudaStream_t s);

}  // namespace iluk
