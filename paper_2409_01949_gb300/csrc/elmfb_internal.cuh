// Internal declarations of the GB300 ELM-FBPINN library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/elmfb.h"

#define ELMFB_LIKELY(x) __builtin_expect(!!(x), 1)

// ---------------------------------------------------------------------------
// error plumbing: every ABI entry point catches elmfb_error and stores the
// message in the handle.
// ---------------------------------------------------------------------------
struct elmfb_error {
  int code;
  std::string msg;
};

#define ELMFB_THROW(code, msg) throw elmfb_error{(code), (msg)}
#define CUDA_CHECK(call)                                                          \
  do {                                                                            \
    cudaError_t e__ = (call);                                                     \
    if (e__ != cudaSuccess)                                                       \
      throw elmfb_error{e__ == cudaErrorMemoryAllocation ? ELMFB_ERR_OOM : ELMFB_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e__)};     \
  } while (0)

// The library's stream-ordered memory pool on the current device.  Freed
// blocks stay cached in it (release threshold: never), so that handles made
// one after another reuse device memory instead of returning it to the system
// at every stream synchronisation; elmfb_trim_memory() hands it back.
cudaMemPool_t library_pool();

// ---------------------------------------------------------------------------
// device buffer owned by the handle (stream-ordered allocation)
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t n, cudaStream_t stream) {
    if (n <= bytes && p) return;
    release();
    s = stream;
    if (n == 0) return;
    CUDA_CHECK(cudaMallocFromPoolAsync(&p, n, library_pool(), stream));
    bytes = n;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Row padding of a cell of the common refinement and the row-class limit.
constexpr int kCellPad = 16;            // cell row groups are padded to this multiple
constexpr int kMaxClasses = ELMFB_MAX_ROWSETS;

// Row class (interior or boundary set): operator coefficients and row scale
// already divided by L.
struct RowClass {
  double c0, c1[2], c2[2];
  double scale;   // row scale / L (entries of M)
  double hscale;  // row scale (entries of h)
};

// Per-subdomain geometry as used on the device.
struct SubGeom {
  double mu[2];
  double sigma_d[2];      // half-width sigma
  double inv_sigma_d[2];  // 1 / sigma in FP64
  float inv_sigma[2];     // 1 / sigma in FP32
  int level;
  int pad_;
};

// Hard-constraint ansatz of paper §4.3: A(x) = prod_i tanh(w (x_i - lo_i))
// tanh(w (hi_i - x_i)) and its first and second derivative along each axis
// (FP64); w = 0 means no ansatz (A = 1).
struct Ansatz {
  double w;
  double lo[2], hi[2];
};
__host__ __device__ inline Ansatz make_ansatz(const elmfb_config& c) {
  Ansatz a{c.ansatz_omega, {c.lo[0], c.dim > 1 ? c.lo[1] : 0.0},
           {c.hi[0], c.dim > 1 ? c.hi[1] : 1.0}};
  return a;
}
__device__ __forceinline__ void ansatz_at(const Ansatz& an, const double* x, int dim, double& A,
                                          double dA[2], double ddA[2]) {
  double f[2] = {1.0, 1.0}, fp[2] = {0.0, 0.0}, fpp[2] = {0.0, 0.0};
  for (int i = 0; i < dim; ++i) {
    // a = tanh(w (x - lo)), b = tanh(w (hi - x)); (ab)' = a'b + ab', (ab)'' =
    // a''b + 2a'b' + ab'' with a' = w (1 - a^2), a'' = -2 w^2 a (1 - a^2) and
    // b' = -w (1 - b^2), b'' = -2 w^2 b (1 - b^2)
    const double a = tanh(an.w * (x[i] - an.lo[i]));
    const double b = tanh(an.w * (an.hi[i] - x[i]));
    const double ta = 1.0 - a * a, tb = 1.0 - b * b;
    const double a1 = an.w * ta, b1 = -an.w * tb;
    const double a2 = -2.0 * an.w * an.w * a * ta, b2 = -2.0 * an.w * an.w * b * tb;
    f[i] = a * b;
    fp[i] = a1 * b + a * b1;
    fpp[i] = a2 * b + 2.0 * a1 * b1 + a * b2;
  }
  A = f[0] * f[1];
  dA[0] = fp[0] * f[1];
  dA[1] = f[0] * fp[1];
  ddA[0] = fpp[0] * f[1];
  ddA[1] = f[0] * fpp[1];
}

struct Stage {
  cudaEvent_t a = nullptr, b = nullptr;
};

// kernels with device timing (elmfb_kernel_stats)
enum KernelId {
  KID_ASSEMBLE = 0, KID_GATHER, KID_ENTRY_T, KID_PANEL_T, KID_PRECOND, KID_UPDATE,
  KID_GRAM_DIAG, KID_BLOCK_CHOL, KID_GRAM_TC, KID_CELL_SORT, KID_FUSED, KID_GSPMV, KID_COUNT
};
struct ProfRec {
  int kid;
  cudaEvent_t a, b;
  int64_t seq;   // the kernel's launch ordinal (prof_seen before this launch)
};

struct elmfb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  elmfb_config cfg{};
  std::string err;
  int64_t launches = 0;

  // geometry (host)
  int dim = 1, L = 1, K = 1, n_sub = 0;
  int64_t NPhi = 0;
  std::vector<int> lev_n, lev_sub_off;  // [L], [L+1]
  std::vector<SubGeom> sub;             // [n_sub]
  std::vector<int> param_sub;           // per subdomain: the full-grid subdomain whose draws it takes
  std::vector<double> bnd[2];           // cell boundaries per dimension
  int nc[2] = {1, 1};
  int n_cells = 0;
  std::vector<int> sub_c0[2], sub_c1[2];  // [n_sub] cell range per dimension
  std::vector<int> cover_off;             // [n_cells+1]
  std::vector<int> cover_sub;             // [n_entries] covering subdomains per cell
  std::vector<int> cell_level_off;        // [n_cells*(L+1)]
  int max_cover = 0;

  // device copies of the geometry
  DevBuf d_sub, d_W32, d_b32, d_W64, d_b64, d_bnd, d_cover_off, d_cover_sub, d_cell_level_off;

  // assembled system
  bool assembled = false;
  int n_classes = 0;
  RowClass cls[kMaxClasses];
  int64_t n_rows = 0;           // user rows
  int64_t NR = 0;               // padded sorted rows
  int64_t NPR = 0;              // panel rows (padded)
  int64_t nnz = 0;
  std::vector<int> cell_count, cell_pstart;   // [n_cells], [n_cells+1]
  std::vector<int64_t> panel_off;             // [n_sub+1]
  std::vector<int> cover_start;               // [n_entries] panel-local first row of the cell
  std::vector<int> row_class_of_set;          // per user row set: class id
  int64_t n_gram_pairs = 0;
  double gram_flops = 0.0;

  DevBuf d_pts_user, d_rhs_user, d_cls_user;  // user order
  DevBuf d_cls;                                 // [kMaxClasses] RowClass table
  DevBuf d_row_cell, d_cell_count, d_cell_pstart;
  DevBuf d_sorted;      // [NR] user row of each sorted row (-1 = padding)
  DevBuf d_x;           // [NR*dim] coordinates (sorted order)
  DevBuf d_rcls;        // [NR] class (sorted order; -1 padding)
  DevBuf d_h;           // [NR] scaled rhs (sorted order)
  DevBuf d_grow_cell;   // [NR] cell of each sorted row
  DevBuf d_u2s;         // [n_rows] sorted position of each user row
  DevBuf d_cover_start, d_panel_off;   // per-panel row numbering (BF16 copy, Gram pairs)
  // Panel storage is cell-interleaved: the rows of cell c start at element row
  // cell_eoff[c]; row p holds the K entries of each of the cell's m_c covering
  // panels in turn, so entry e = (c, panel w) row p sits at element row
  // entry_base[e] + p m_c with entry_base[e] = cell_eoff[c] + w.
  std::vector<int64_t> cell_eoff, entry_base;
  DevBuf d_cell_eoff, d_entry_base;
  DevBuf d_panels;      // [NPR*K] FP64, FP32 or FP32 pairs
  DevBuf d_tiles;       // per-panel tiles: (entry, first row) of 32 rows
  int64_t n_tiles = -1;  // -1 until the QR needs them (ensure_qr_tiles)
  DevBuf d_ltiles;      // assembly tiles: (first entry of a level group, entries, first row)
  int64_t n_ltiles = 0;
  int nl_max = 1;       // most covering entries of one level in one cell
  std::vector<int> entry_cell;   // [n_entries]
  DevBuf d_entry_cell;
  DevBuf d_flags;       // device status flags (int[4])

  // BF16 feature-major panel copy PT[k][rho] (mixed precision) and Gram blocks
  DevBuf d_pt;
  std::vector<std::pair<int, int>> gram_pair_ij;   // sorted (i <= j)
  int64_t gram_runs = 0;
  DevBuf d_gram_pairs, d_gram_runs, d_gram;        // d_gram: [pair][K][K] FP32
  bool have_gram = false;

  // learned preconditioner: subdomain graph, weights, Adam moments, work buffers
  std::vector<int> gnn_off, gnn_nb;
  DevBuf d_gnn_off, d_gnn_nb, d_gnn_w, d_gnn_m, d_gnn_v, d_gnn_act, d_gnn_lp, d_gnn_dy;
  bool gnn_trained = false;

  // Golub-Kahan record of the last LSQR solve: alpha_1.., beta_1..
  std::vector<double> gk_alpha, gk_beta;

  // solution
  DevBuf d_a;           // [NPhi] FP64
  bool have_coeffs = false;

  // solver work buffers
  DevBuf d_u, d_v, d_w, d_x_sol, d_tmp, d_partial, d_scal, d_R, d_ptile, d_gpart;
  DevBuf d_R2;   // X_j as FP32 pairs, packed lower triangle per panel (FP32 and DF32 panels)

  // stage timers
  Stage st[ELMFB_N_STAGES];
  double stage_ms[ELMFB_N_STAGES] = {0};

  // per-kernel profiling
  bool prof = false;
  uint64_t prof_mask = ~uint64_t(0);   // kernels timed when prof is on (bit = KernelId)
  std::vector<ProfRec> prof_live;       // recorded, not yet harvested
  std::vector<cudaEvent_t> prof_pool;   // free events
  double prof_ms[KID_COUNT] = {0};
  int64_t prof_n[KID_COUNT] = {0};
  double prof_bytes[KID_COUNT] = {0};   // algorithmic bytes per launch (last launch)
  int prof_stride = 1;                  // time every prof_stride-th launch of a kernel
  int bj_retries = 0;                   // block-Jacobi factorisations redone with a larger shift
  int bj_dropped = 0;                   // block-Jacobi columns dropped as dependent
  int64_t prof_seen[KID_COUNT] = {0};   // launches seen while profiling
  bool prof_now[KID_COUNT] = {false};   // the current launch carries events

  // ELMFB_FP32_DF32: d_panels holds the FP32 panels, d_panels_df the pairs
  DevBuf d_panels_df;
  bool bj_reuse = false;   // LSQR refinement: keep the block-Jacobi factors of the last set-up
  // batched graphs: a device flag the LSQR loop's kernels read first (nonzero:
  // return at once); null outside a batched graph
  struct BatchRound* round = nullptr;   // the batch's coordinator (batch.cu), or null
  bool blocking_sync = false;   // waits sleep on an event (batch workers) instead of spinning
  bool tune_lookup_only = false;   // autotune: use recorded choices only (concurrent batch)
  cudaEvent_t sync_ev = nullptr;
  int round_slot = -1;
  bool dual() const { return cfg.precision == ELMFB_FP32_DF32; }
  bool fp64() const { return cfg.precision == ELMFB_FP64; }
  bool df32() const { return cfg.precision == ELMFB_DF32; }
  // entries evaluated in FP64 (FP64 panels, or FP32 pairs split from FP64)
  bool eval64() const { return fp64() || df32(); }
  size_t panel_elem() const { return eval64() ? 8 : 4; }
};

// stage timing helpers
void stage_begin(elmfb_ctx* h, int s);
void stage_end(elmfb_ctx* h, int s);   // records; time read lazily
void stage_collect(elmfb_ctx* h);

// assembly (assemble.cu)
void assemble_system(elmfb_ctx* h, int n_sets, const elmfb_rowset* sets);
// out = the items (ent[g], rows t), t < off[g + 1] - off[g], of every group g in
// order, written on the device (int2; off[0] = 0)
void expand_entry_steps(elmfb_ctx* h, const std::vector<int>& ent, const std::vector<int64_t>& off,
                        int rows, DevBuf& out);
void ensure_qr_tiles(elmfb_ctx* h);   // h->d_tiles / n_tiles for the QR's densification
void export_rows(elmfb_ctx* h, const int64_t* rows, int64_t n, double* out, double* h_out);

// tensor-core Gram (gram_tc.cu)
void gram_build_pairs(elmfb_ctx* h);
void gram_compute(elmfb_ctx* h);

// solve (solve.cu)
void solve_system(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info);
// extreme singular values of the Golub-Kahan bidiagonal recorded as (alpha,
// beta) pairs, k steps: out2[0] = sigma_max, out2[1] = sigma_min (device)
void bidiag_extremes(elmfb_ctx* h, const double* gk, int k, double* out2);
// dense column-pivoted QR solve (direct.cu)
void qr_solve(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info);

// Work plan of the fused pass: units (cell, row range, first partial) and, per
// panel, the list of partial rows that sum to its part of M^T u'.
// Panel element of ELMFB_DF32: an FP32 pair, value hi + lo (|lo| <= ulp(hi)/2).
struct __align__(8) df2 {
  float hi, lo;
};

struct FusedPlan {
  DevBuf units, fo, fe, part;
  DevBuf tf;            // FP32 copy of t for FP32 panels
  DevBuf pch, pco, csum;   // per-panel slices of the partial list and their sums
  int n_pchunks = 0;
  int n_units = 0;
  int max_unit_rows = 0;   // rows of the largest unit (its u values are staged in smem)
  int threads = 0;
  bool pairs = false;   // partials are FP32 (hi, lo) pairs, value hi - lo
};
// unit_rows >= 8 forces the rows per work unit (the autotuner's choice)
bool build_fused_plan(elmfb_ctx* h, FusedPlan& fp, int unit_rows = 0);
int64_t fused_unit_target(const elmfb_ctx* h);
// mode 0: u' = M t - (alpha/beta) u (staged alpha, beta); mode 1: u' = h - M t;
// mode 2: u' = (M t) s - (alpha/beta) u with s the staged 1/alpha (t = P v',
// v' = alpha v not yet normalised).
// Writes u', per-panel partials of M^T u' into fp.part (FP64 values for FP64
// panels; compensated FP32 (hi, lo) pairs in the same 8 bytes for FP32
// panels) and ||u'||^2 per unit.  tf: FP32 copy of t (FP32 panels) or FP32
// pairs (DF32 panels), or null to convert t here.
template <class T>
void launch_fused(elmfb_ctx* h, FusedPlan& fp, const double* t, int mode, double* scal,
                  double* gpart, const void* tf = nullptr);
template <class T>
void block_jacobi_setup(elmfb_ctx* h, double shift, bool identity, double abs_shift = 0.0,
                        double drop = 0.0);
// fixed slices of each panel's partials; with beta_partial (LSQR) also the
// commit of the staged scalars and beta^2 into the staged slot that the panel
// kernels read
void panel_chunk_sums(elmfb_ctx* h, FusedPlan& fp, const double* beta_partial = nullptr,
                      int n_beta = 0, double* scal = nullptr);
void panel_sum(elmfb_ctx* h, FusedPlan& fp, double* g);               // g_s = sum of partials
void bj_apply(elmfb_ctx* h, const double* r, double* z, double* dot_part);  // z = X^T X r

// Multi-instance LSQR launches (batch.cu): the instances of
// elmfb_batch_solve that iterate on FP32 panels with the FP32-pair tail join
// shared rounds; one round runs check_every LSQR iterations of every member,
// each iteration as three launches per launch shape (the fused pass, the
// slice sums, the tail) whose blocks map to (member, local unit / slice /
// panel) and read that member's arrays from its BatchInst.  Every block does
// exactly what it does in the instance's own launch, so each instance's
// iterates are bitwise those of solving it alone.
struct BatchInst {
  // fused pass
  const float* panels;
  const float* tlow;   // FP32 copy of t
  const int4* units;
  const int* cell_pstart;
  const int* cell_count;
  const int* cover_off;
  const int* cover_sub;
  const int64_t* entry_base;
  double* scal;
  double* u;
  const double* hvec;
  double* part;
  double* gpart;   // per-unit ||u'||^2 partials
  int* flags;
  // slice sums
  const int* fe;
  const int2* pch;
  double* csum;
  // tail
  const int* pco;
  const float2* Xt;
  double* v;
  double* w;
  double* x;
  double* vpart;   // per-panel ||v'||^2 partials
  double* t;
  unsigned int* counter;
  int n_units, n_pchunks, n_sub, pad_;
};
// What the members of one multi-instance launch must share.
struct BatchShape {
  int K = 0, fpl = 0, rows = 0, S = 0, mmax = 0, pthreads = 0, chunk_threads = 0, low_kind = 0,
      mode = 0, tthreads = 0;
  size_t smem = 0, tsmem = 0;
  bool operator<(const BatchShape& o) const {
    const int a[10] = {K, fpl, rows, S, mmax, pthreads, chunk_threads, low_kind, mode, tthreads};
    const int b[10] = {o.K, o.fpl, o.rows, o.S, o.mmax, o.pthreads, o.chunk_threads, o.low_kind,
                       o.mode, o.tthreads};
    for (int i = 0; i < 10; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    if (smem != o.smem) return smem < o.smem;
    return tsmem < o.tsmem;
  }
};
struct BatchRound;
// The staged LSQR scalars and the first four flags of one member after a
// round, as the coordinator gathers them for all members at once.
constexpr int kRoundRecord = 28;   // 24 staged scalars, 4 flags
// join with the instance's arrays; then round_step() once per check interval
// (fills rec with this member's record; returns the shared launches
// attributed to it, each launch to one member); round_leave() when done
void round_join(BatchRound* r, int slot, const BatchInst& inst, const BatchShape& shape);
int64_t round_step(BatchRound* r, int slot, double* rec);
void round_leave(BatchRound* r, int slot);
int round_interval(const BatchRound* r);   // iterations per round
// one LSQR iteration of a launch shape's members: n_f units, n_c slices, n_t
// panels over all of them (solve.cu)
void launch_batch_iteration(const BatchShape& sh, const BatchInst* d_inst, const int2* d_fmap,
                            int n_f, const int2* d_cmap, int n_c, const int2* d_tmap, int n_t,
                            cudaStream_t st);
// out[j] = member j's record (kRoundRecord doubles) from its scal and flags
void launch_gather_records(const BatchInst* d_inst, int n, double* out, cudaStream_t st);

// learned preconditioner (gnn.cu)
void fcg_solve(elmfb_ctx* h, const elmfb_solve_opts* o, elmfb_solve_info* info);

// coarse-level correction of block-Jacobi (coarse.cu): the joint block of the
// columns of levels 1..levels
int coarse_columns(const elmfb_ctx* h, int levels);
void coarse_setup(elmfb_ctx* h, int levels, double shift,
                  const std::function<void(const double*, double*)>& normal_op, DevBuf& X,
                  int* retries);
void coarse_apply(elmfb_ctx* h, const DevBuf& X, int n, const double* r, double* z, DevBuf& tmp);

// eval (eval.cu)
void eval_model(elmfb_ctx* h, const double* xs, int64_t n, double* out);
void error_norms(elmfb_ctx* h, const double* uh, const double* ur, int64_t n, double* out3);

// per-kernel profiling (no-ops when h->prof is false)
void prof_begin(elmfb_ctx* h, int kid, double bytes);
void prof_end(elmfb_ctx* h, int kid);
void prof_harvest(elmfb_ctx* h, size_t keep = 0);   // all but the last `keep` records
// forget the timed launches of kernel kid from ordinal `from` on (launches
// that returned at once after LSQR stopped on the device)
void prof_drop_from(elmfb_ctx* h, int kid, int64_t from);

// helpers
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline void count_launch(elmfb_ctx* h, int n = 1) { h->launches += n; }
void check_launch(const char* what);
int64_t count_gram_pairs(const elmfb_ctx* h);   // pairs (i <= j) sharing a cell with points
// Raise, never lower, a kernel's dynamic shared-memory limit on the current
// device.  The attribute is process-wide, so handles solving concurrently in
// other threads only ever see it grow.
void ensure_dyn_smem(const void* func, size_t bytes, bool max_carveout = false);
// Wait for the handle's stream: cudaStreamSynchronize, or with blocking_sync
// an event recorded on it and waited on with blocking synchronisation (the
// thread sleeps: a batch runs more host threads than cores, and spinning
// waiters starve the threads with work to do).
void stream_sync(elmfb_ctx* h);
