// internal.cuh -- declarations shared by the library's translation units.
//
// Nothing here is part of the public ABI (include/sphynx.h).  Errors inside
// the library are C++ exceptions of type sphynx::Error; every extern "C"
// entry point catches them and returns the status code.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/sphynx.h"

namespace sphynx {

struct Error {
  int code;
};

[[noreturn]] void fail(int code, const char *fmt, ...);
[[noreturn]] void fail_cuda(cudaError_t e, const char *what, const char *file, int line);
void set_error_message(const char *msg);
void clear_error();

#define SPX_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) ::sphynx::fail_cuda(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SPX_LAUNCHED() SPX_CUDA(cudaGetLastError())

// Runs `body` and converts exceptions into status codes at the ABI boundary.
template <class F>
int guarded(F &&body) {
  try {
    clear_error();
    return body();
  } catch (const Error &e) {
    return e.code;
  } catch (...) {
    set_error_message("unexpected C++ exception");
    return SPHYNX_ERR_CUDA;
  }
}

// Owning device allocation.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    release();
    p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0;
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t nbytes);   // throws OOM; contents undefined
  void release();
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// Block element types used by the kernels.
enum class DT { F64 = SPHYNX_DT_F64, F32 = SPHYNX_DT_F32, BF16 = SPHYNX_DT_BF16 };
inline size_t dt_size(DT d) { return d == DT::F64 ? 8 : (d == DT::F32 ? 4 : 2); }

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based
// generator: draw ctr (>= 1) of the stream that starts at `state`.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// u in [0,1) from the top 53 bits, then 2u - 1 (exact in double)
__device__ inline double splitmix_pm1(uint64_t state, uint64_t ctr) {
  const uint64_t z = mix64(state + ctr * kGamma);
  return 2.0 * (static_cast<double>(z >> 11) * 0x1.0p-53) - 1.0;
}

constexpr int kShortDeg = 32;        // rows with more neighbours are medium or long rows
constexpr int kMedDeg = 4096;        // rows with more neighbours than this are long rows
constexpr int kGroupPerLane = 16;    // medium rows: entries a lane of a row's group takes at most (G < 32)
constexpr int kLongChunk = 1024;     // entries per long-row work item (32 a lane: short gather chains)
constexpr int kSmCount = 152;

// Short-row schedules the autotuner chooses between.
enum SpmmVariant : int {
  kCsrStaged = 0,   // CSR: a warp stages its 32 rows' columns in shared memory
  kSell32 = 1,      // SELL-32: columns stored slice-major, read straight from global memory
  kSellPattern = 2, // SELL-32 whose shared-pattern slices store one offset list per slice
};
constexpr int kSpmmVariants = 3;
// sell_cptr / pat_cptr tag of a shared-pattern slice (the start follows in the low bits)
constexpr int64_t kPatternTag = int64_t{1} << 62;

constexpr int kSellLsCount = 5;      // slice strides 1, 2, 4, 8, 16 the autotuner times

struct SpmmTuning {
  int variant;
  float us[kSpmmVariants];           // measured time of each schedule (1e30: not available)
};

struct SpmmPlan {
  int variant = kCsrStaged;          // schedule of the launch being issued
  int forced = -1;                   // >= 0: every product uses this schedule
  int tuned_variant = kCsrStaged;    // the autotuner's choice for this graph
  float tuned_us[kSpmmVariants] = {0.f, 0.f, 0.f};   // its timings of the schedules
  int sell_ls = 0;                   // SELL blocks: warps take slices 2^sell_ls apart
  float tuned_ls_us[kSellLsCount] = {};   // the autotuner's time for each sell_ls
  DevBuf tune_scratch;
  int64_t n_long = 0;                // long rows: degree > kMedDeg
  int64_t n_items = 0;               // long-row work items
  DevBuf items;                      // int64 [n_items][4]: row, begin, end, slot
  DevBuf split;                      // int64 [n_long][3]: row, first slot, slot count
  DevBuf partials;                   // per-item partial rows (n_items x 16 doubles)
  // SELL-32 copy of the short rows.  Slice s (rows 32s..32s+31) holds entry t
  // of its lane-th row at position 32 t + lane of its block.  A slice whose
  // entries all lie within 32767 of their row stores 16-bit offsets col - row,
  // any other slice 32-bit column indices; sell_cptr[s] is the block's start
  // in 16-bit units, bitwise negated for a 16-bit slice.  Weights, when
  // present, are at sell_w[sell_ptr[s] + 32 t + lane].
  int64_t sell_entries = 0;          // padded entries of all slices
  int64_t sell_narrow = 0;           // slices stored with 16-bit offsets
  double short_entries = 0;          // entries of the rows with at most kShortDeg neighbours
  double sell_bytes = 0;             // bytes a product must read from this layout:
                                     // real entries' indices, degrees, slice offsets
  DevBuf sell_ptr;                   // int64 [n_slices + 1], entry offsets
  DevBuf sell_cptr;                  // int64 [n_slices], see above
  DevBuf sell_col;                   // 16-bit units [sum of block sizes]
  DevBuf sell_w;                     // float [sell_entries] (weighted graphs)
  DevBuf sell_deg;                   // uint8 [n]: degree, or 0xFF for a long row
  // Shared-pattern slices (unweighted graphs): a slice whose 32 rows' short-row
  // offsets col - row take at most 31 distinct values, all within 16 bits,
  // stores that sorted union U once (32 int16, zero padded: 64 bytes) and one
  // 32-bit mask per row (128 bytes): bit k says the row has the entry
  // row + U[k], bit 31 marks a lane without a short row (a long row or a
  // padding lane).  A row's entries in mask order are its CSR entries in
  // order, so its sum is the explicit slice's sum.  pat_cptr[s] is
  // kPatternTag | (start in pat_col, 16-bit units) for such a slice and
  // sell_cptr[s] (the explicit slice in sell_col) for the others.
  int64_t pat_slices = 0;            // shared-pattern slices (0: the variant is not built)
  bool pat_all = false;              // every slice is a shared-pattern slice
  // Normalized products with float or double input gather rows of
  // Z = D^{-1/2} X, formed by one pass before the product, instead of X rows
  // and the neighbour's D^{-1/2} entry: on an irregular graph that second
  // gather costs a 32-byte sector per entry.  Set at create for irregular
  // graphs (maximum degree above 10 x the mean).
  bool prescale = false;
  // Normalized products with bfloat16 input on irregular graphs read a
  // per-entry coefficient c_ij = (w_ij or 1) D^{-1/2}_j, rounded in float as
  // the kernels round it, from a stream (CSR order and SELL slot order)
  // instead of gathering D^{-1/2}_j; built at the first such product.
  DevBuf ncoef_csr;                  // float [nnz]
  DevBuf ncoef_sell;                 // float [sell_entries]
  double pat_bytes = 0;              // bytes a product reads from this layout
  DevBuf pat_cptr;                   // int64 [n_slices]
  DevBuf pat_col;                    // 16-bit units, 96 per shared-pattern slice
  double long_bytes = 0;             // bytes of the long rows' CSR entries and items
  // Medium rows (kShortDeg < degree <= med_max), sorted by degree (descending,
  // row id on ties) into grp_row, and cut into warp units of rows that share
  // a group width G (a power of two, G lanes per row): unit u covers rows
  // grp_row[x .. x + count) with {x, log2 G | count << 8} = grp_unit[u].  Their
  // entries are read from the graph's own CSR arrays.
  int med_max = kMedDeg;             // largest degree of a medium row (the autotuner's choice)
  int64_t n_med = 0, n_units = 0;
  DevBuf grp_row;                    // int32 [n_med]
  DevBuf grp_unit;                   // int2 [n_units]
  double med_bytes = 0;              // bytes a product reads for the medium rows
};

// Everything the iteration kernels need to apply L without forming it.
struct LapView {
  int64_t n;
  const int64_t *rowptr;
  const int32_t *col;
  const float *w;          // NULL = unit weights
  const double *deg;       // weighted degree (double)
  const float *degf;       // weighted degree (float)
  const double *dinv;      // deg^{-1/2}
  const float *dinvf;
  int gather_scale;        // normalized: scale gathered rows by dinv (0: the input is D^{-1/2} X already)
};

struct Counters {
  int64_t launches = 0;
  int64_t spmm_launches = 0;
  double spmm_bytes = 0;
  double spmm_ms = 0;
  // the same split by input precision (indexed by DT)
  int64_t spmm_launches_dt[3] = {0, 0, 0};
  double spmm_bytes_dt[3] = {0, 0, 0};
  double spmm_ms_dt[3] = {0, 0, 0};
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;  // pairs recorded around SpMMs
  std::vector<int> ev_dt;            // input precision of each recorded pair
  size_t ev_used = 0;
};

// A batch of graphs in one handle (sphynx_create_batch): graph q owns rows
// [h_gptr[q], h_gptr[q+1]); row-reducing kernels work on chunks of rows that
// never straddle two graphs.
struct BatchInfo {
  int count = 0;                    // 0: the handle holds one graph
  std::vector<int64_t> h_gptr;      // [count + 1] graph offsets (host)
  DevBuf gptr;                      // the same on the device
  int64_t n_chunks = 0;
  DevBuf chunk_graph;               // int32 [n_chunks]: graph of each chunk
  DevBuf chunk_begin;               // int64 [n_chunks + 1]: first row of each chunk, then n
  DevBuf graph_chunk0;              // int32 [count + 1]: first chunk of each graph
  DevBuf graph_max;                 // uint64 [count][2]: max degree, max weighted degree (double bits)
  DevBuf row_graph;                 // int32 [n]: graph of every row (the chain reads its roots)
  // rows in reverse Cuthill-McKee order within each graph (batches created
  // from host arrays): orig[r] = the caller's vertex at internal row r, and
  // the caller's vertex weights in the caller's order (multi-jagged runs there)
  DevBuf orig;                      // int32 [n], empty: the caller's order
  DevBuf vw_orig;                   // int64 [n] (vertex-weighted batches)
  // while a batched eigensolve runs: the 1024-row blocks and the chunks that
  // hold rows of graphs still iterating (rebuilt after every convergence
  // test), and their counts [blocks, chunks]; the products and the chunk
  // kernels walk these lists with fixed grids, so finished graphs cost nothing
  DevBuf act_blocks, act_chunks, n_act;
  // polynomial preconditioner of every graph (Sec. 5.2), set up per partition
  int poly_k = 0;                   // chain length: the largest root count of any graph (0: none set up)
  int poly_lap = -1;
  DevBuf poly_inv;                  // double [count][poly_k + 1]: 1 / theta in application order, then 0
  DevBuf poly_invf;                 // float copy
};

// aggregation multigrid hierarchy (amg.cu), owned by the handle
struct AmgHierarchy;
void amg_free(AmgHierarchy *h);

}  // namespace sphynx

struct sphynx_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0, nnz = 0;
  bool weighted = false, has_vw = false;
  const int64_t *rowptr = nullptr;
  const int32_t *col = nullptr;
  const float *w = nullptr;
  const int64_t *vw = nullptr;
  sphynx::DevBuf own_rowptr, own_col, own_w, own_vw;
  sphynx::DevBuf deg, degf, dinv, dinvf;
  sphynx::DevBuf jinv, jinvf;  // Jacobi: 1 / deg (1 where deg = 0)
  int64_t max_degree = 0;
  double max_wdeg = 0;
  int64_t total_vw = 0;
  int64_t isolated = 0;
  int wscale = 0;            // exact-cut fixed point: weight * 2^wscale is an integer
  bool wexact = true;        // the fixed-point sum cannot overflow int64
  sphynx::SpmmPlan plan;
  // polynomial preconditioner state (Sec. 5.2)
  int poly_k = 0;            // roots (degree plus definiteness copies)
  int poly_degree = 0;       // the degree it was set up for
  int poly_laplacian = -1;
  sphynx::DevBuf poly_inv;   // double[k + 1]: 1 / theta_i, then 0
  sphynx::DevBuf poly_invf;  // float[k + 1]
  std::vector<double> poly_roots;
  double step_theta[2] = {0.0, 0.0};         // roots whose reciprocals sphynx_poly_step last uploaded
  std::map<std::string, sphynx::DevBuf> ws;  // named workspaces, grown on demand
  sphynx::Counters ctr;
  sphynx::DevBuf pinned_dummy;
  void *host_flag = nullptr;                 // pinned int32[8] for convergence polls
  sphynx::BatchInfo batch;                   // set by sphynx_create_batch
  sphynx::AmgHierarchy *amg = nullptr;       // multigrid preconditioner (Sec. 5.3), built on demand
  sphynx::LapView view() const {
    return sphynx::LapView{n, rowptr, col, w, deg.as<double>(), degf.as<float>(),
                           dinv.as<double>(), dinvf.as<float>(), 1};
  }
  void *workspace(const std::string &name, size_t bytes, bool zero = false);
};

namespace sphynx {

// ---- spmm.cu ----------------------------------------------------------------
// Y = L X (mode 0) or one step of the polynomial chain (mode 1):
//   t_out = t - (L t) * inv_cur; yacc gathers t * inv_cur and t_out * inv_next
//   as yterms says (see spmm_kernels.cuh)
struct SpmmArgs {
  int lap;                 // SPHYNX_COMBINATORIAL (also generalized) or SPHYNX_NORMALIZED
  DT tin;                  // element type of x
  int ld_x, ld_y;          // leading dimensions (elements)
  int bp;                  // padded width: 1, 4, 8, 12 or 16
  int b_true;              // columns counted as algorithmic bytes
  const void *x;
  void *y;                 // mode 0: double (F64 input) or float
  int mode;                // 0 plain, 1 polynomial step
  void *t_out;             // mode 1: next chain vector, element type tout
  DT tout;                 // mode 1: F64 (with F64 input), F32 or BF16
  void *yacc;              // mode 1: double or float accumulator (ld_y)
  int first;               // mode 1: initialise yacc from t
  int yterms;              // mode 1: terms added to yacc: 2 (t and t'), 1 (t' only) or 0
  const double *inv;       // mode 1: device array of 1/theta
  const float *invf;       // mode 1: its float copy
  int i_cur;               // mode 1: index of theta_i in inv
  const int *done;         // device flag: skip the launch when nonzero (may be NULL)
  const int32_t *row_graph = nullptr;  // batches: graph of each row; in mode 1 its roots
  int inv_stride = 0;                  // are inv[row_graph[row] * inv_stride + i]
  const int32_t *act_blocks = nullptr; // batches: 1024-row blocks holding rows of graphs still
  const int *n_act = nullptr;          // iterating (device list and count); NULL: every row
};
void spmm(sphynx_graph *g, const SpmmArgs &a);
// both short-row schedules timed on this product (scratch outputs)
SpmmTuning spmm_tune(sphynx_graph *g, const SpmmArgs &a);
// every SELL slice stride timed on this product; sets plan.sell_ls to the fastest
void spmm_tune_sell_stride(sphynx_graph *g, const SpmmArgs &a);

// ---- amg.cu -----------------------------------------------------------------
// build the aggregation hierarchy of g (rebuild = false: keep one built for the same seed)
void amg_setup(sphynx_graph *g, int64_t seed, bool rebuild);
// h = one V-cycle applied to the n x ld block r (F32 or F64); launches skip once *done
void amg_apply(sphynx_graph *g, DT dt, const void *r, void *h, int ld, const int *done);
void amg_level_info(sphynx_graph *g, int level, sphynx_amg_level_info *info, int32_t *agg_out, int64_t *rowptr_out,
                    int32_t *col_out, float *w_out);

// ---- dense.cu ---------------------------------------------------------------
void launch_random_block(cudaStream_t s, DT dt, void *x, int64_t n, int b, int ld, uint64_t seed);
void launch_piecewise_block(cudaStream_t s, DT dt, void *x, int64_t n, int b, int ld, int lap,
                            const double *deg);
void launch_from_f64(cudaStream_t s, DT dt, void *x, const double *src, int64_t n, int b, int ld);
void launch_to_f64(cudaStream_t s, DT dt, const void *x, double *dst, int64_t n, int b, int ld);
void launch_zero(cudaStream_t s, void *p, size_t bytes);

struct GramArgs {
  DT dt;                      // F64 or F32
  int nblk, ld;               // S = [blk0 | blk1 | blk2], each ld wide
  int64_t n;
  const void *s[3];
  const void *ls[3];
  const double *bdiag;        // double (F64) -- NULL for B = I
  const float *bdiagf;        // float copy (F32)
  double *partials;           // scratch: gram_partials_size() doubles
  double *ga, *gb;            // M x M outputs (device)
  const int *done;
};
int gram_grid(int64_t n);
size_t gram_partials_size(int nblk, int ld, int grid);
// launches at most `grid` CTAs and returns how many partial rows it wrote
int launch_gram(cudaStream_t st, const GramArgs &a, int grid);

struct UpdateArgs {
  DT dt;
  int nblk, ld;
  int64_t n;
  const void *s[3];          // X, H, P
  const void *ls[3];         // (unused), LH, LP
  const void *y;             // M x ld coefficients in dt
  void *xo, *po, *lpo;       // X' = S Y; P' = [0 H P] Y; LP' = [0 LH LP] Y
  const int *done;
};
void launch_update(cudaStream_t st, const UpdateArgs &a);

struct ResidualArgs {
  DT dt;
  int ld;
  int64_t n;
  const void *x, *lx;
  const double *theta;       // device [ld]
  const double *bdiag;       // B diagonal (double) or NULL
  const float *bdiagf;
  const double *jinv;        // Jacobi inverse diagonal (double) or NULL = no scaling
  const float *jinvf;
  void *out;                 // R or H = Jacobi(R)
  double *norm_partials;     // [grid][ld]
  const int *done;
  int out_bf16 = 0;          // float blocks: out stored in bfloat16 (the mixed chain's first input)
};
int residual_grid(int64_t n);
void launch_residual(cudaStream_t st, const ResidualArgs &a, int grid);

struct SolverState {         // device-resident LOBPCG bookkeeping
  double theta[SPHYNX_MAX_NEV];
  double resnorm[SPHYNX_MAX_NEV];
  int conv[SPHYNX_MAX_NEV];
  int pvalid;
  int done;
  int iters;
  int status;
  int svqb_steps;
  int nconv;
  int stalled;                     // stopped by the stall window
  int pad;
  double best_res[SPHYNX_MAX_NEV]; // smallest residual so far per column (0: none yet)
  int since_best[SPHYNX_MAX_NEV];  // iterations since it last fell below 0.9 x best
};
// Stall window: true once every unconverged column has gone `window`
// iterations without its residual falling below 0.9 x its best so far.
__device__ inline bool stall_check(SolverState *st, int b, int window, int count_iteration, double floor_th) {
  if (window <= 0 || !count_iteration) return false;
  bool all = true;
  for (int j = 0; j < b; ++j) {
    if (st->conv[j]) continue;
    const double r = st->resnorm[j];
    if (st->best_res[j] == 0.0 || r < 0.9 * st->best_res[j]) {
      st->best_res[j] = r;
      st->since_best[j] = 0;
    } else {
      st->since_best[j] += 1;
    }
    // a column still far above the noise floor is converging slowly, not stalled
    all = all && st->since_best[j] >= window && st->best_res[j] <= floor_th;
  }
  return all;
}

void launch_converge(cudaStream_t st, SolverState *state, const double *partials, int grid, int b,
                     int ld, double tol, double floor_th, double floor_res, int count_iteration, int maxit,
                     int stall_window = 0, int abs_test = 0);

void launch_signs_coords(cudaStream_t st, DT dt, const void *x, int64_t n, int ld, int b,
                         void *coords, double *scratch);

// dots and vector ops for the Lanczos process of the polynomial setup
// The basis is column-major (column c at basis + c * ldv, ldv a multiple of 4,
// basis and w 32-byte aligned); partials hold grid x j1 doubles.
void launch_lanczos_dots(cudaStream_t st, DT dt, const void *basis, int64_t ldv, int j1,
                         const void *w, int64_t n, double *partials, int grid);
void launch_reduce_cols(cudaStream_t st, const double *partials, int grid, int cols, double *out);
void launch_lanczos_sub(cudaStream_t st, DT dt, const void *basis, int64_t ldv, int j1, void *w,
                        int64_t n, const double *h, double *norm_partials, int grid);
void launch_lanczos_next(cudaStream_t st, DT dt, const void *w, void *v, void *basis, int64_t ldv,
                         int j, int64_t n, const double *beta2);
void launch_poly_start(cudaStream_t st, DT dt, void *v, int64_t n, uint64_t seed);
void launch_project_null(cudaStream_t st, DT dt, void *v, int64_t n, int lap, const double *deg,
                         double *partials, int grid, double *scal);
// option checks shared by the single-graph and batched solvers
void check_lobpcg_options(const sphynx_graph *g, const sphynx_options *o);
// The embedding's canonical rotation on the rows x[0..rows) (ld wide, d
// eigenvectors, Ritz values theta): within every run of Ritz values closer
// than tol, the columns are turned to their orthogonal Procrustes alignment
// with the seeded reference block (lobpcg.cu).
void canonical_rotation_block(sphynx_graph *g, void *x, int64_t rows, int ld, DT dt, const double *theta, int d,
                              double tol, uint64_t seed);
// Canonical rotation of a cluster of eigenvectors (columns a .. a + c - 1 of
// the n x ld block x, d eigenvectors): partials[grid][c] of row p of
// E_c^T Z_c, Z the reference block drawn from mix64(seed + 5 gamma) with
// counter i * d + j + 1; and E_c <- E_c Q for a device c x c row-major Q.
void launch_cluster_dots(cudaStream_t st, DT dt, const void *x, int64_t n, int ld, int d, int a, int c, int p,
                         uint64_t seed, double *partials, int grid);
void launch_rotate_cols(cudaStream_t st, DT dt, void *x, int64_t n, int ld, int a, int c, const double *q);
// col = z / ||z||, z the null vector of L (1, or D^{1/2} 1 for L_N), with
// scal[1] = z . z as launch_project_null leaves it
void launch_null_column(cudaStream_t st, DT dt, void *col, int64_t n, int lap, const double *deg,
                        const double *scal);
void launch_poly_single(cudaStream_t st, DT dt, const void *r, void *h, int64_t n, int ld,
                        const double *inv, const int *done);
int vec_grid(int64_t n);

// ---- small.cu ---------------------------------------------------------------
// M x M Gram matrices; coefficients written as M x ld (ld >= b); without an
// active mask, column k of S is block k / ld, column k % ld.  mixed: the
// FP64 symmetric eigen-solves start from a float Jacobi basis (the result is
// still the double solve's; see eig_sym).  count > 1 solves that many
// problems, laid out back to back in every array, one CTA each.
void launch_rayleigh_ritz(cudaStream_t st, const double *ga, const double *gb, int M, int ld,
                          int b, double u_work, SolverState *state, double *y64, void *yt, DT dt,
                          const int *active_override, double *theta_out, int *svqb_out, int mixed,
                          int count = 1);
void launch_d2f(cudaStream_t st, const double *src, float *dst, int64_t n);
void launch_gram_reduce(cudaStream_t st, const double *partials, int nblk, int ld, int grid,
                        double *ga, double *gb, const int *done);
// Roots of the degree-k GMRES polynomial in application order, with the
// definiteness copies: kout receives the count k' <= k + SPHYNX_MAX_ADDED_ROOTS;
// roots[k' .. k + SPHYNX_MAX_ADDED_ROOTS) = +inf, inv / invf = 1 / roots then 0
// up to index k + SPHYNX_MAX_ADDED_ROOTS.
// a reordered batch (sphynx_create_batch from host arrays): p_rows[r] =
// p_caller[orig[r]] on the handle's stream (device arrays of n)
void batch_parts_to_rows(sphynx_graph *g, const int32_t *p_caller, int32_t *p_rows);
void launch_harmonic_ritz(cudaStream_t st, const double *alpha, const double *beta2, int k,
                          double *roots, double *inv, float *invf, int *err, int *kout);
// count problems, problem q's arrays `stride` (>= k + SPHYNX_MAX_ADDED_ROOTS + 1) apart, err and kout [count]
void launch_harmonic_ritz_batch(cudaStream_t st, const double *alpha, const double *beta2, int k, int count,
                                int stride, double *roots, double *inv, float *invf, int *err, int *kout);

// ---- mj.cu ------------------------------------------------------------------
void run_mj(cudaStream_t st, DT dt, const void *coords, int ldc, int dims, int64_t n,
            const int64_t *vw, int K, int32_t *part, Counters *ctr);
// Multi-jagged with caller-provided scratch (mj_scratch_bytes).  With count > 1
// the points are count graphs, graph g owning points [h_gptr[g], h_gptr[g+1])
// (host offsets) and parts [g K/count, (g+1) K/count): the first level has one
// section per graph and every later level splits within them.
size_t mj_scratch_bytes(int64_t n, int K, int count);
void run_mj_scratch(cudaStream_t st, DT dt, const void *coords, int ldc, int dims, int64_t n,
                    const int64_t *vw, int K, int32_t *part, Counters *ctr, void *scratch,
                    const int64_t *h_gptr, int count);

// ---- refine.cu --------------------------------------------------------------
constexpr int kRefineMaxDegree = 256;   // vertices with more neighbours never move
// greedy refinement of the device partition `part` in place (refine.cu)
void refine_partition(sphynx_graph *g, int32_t *part, int K, double eps, int max_rounds, int max_degree,
                      int *moves_out, int *rounds_out);

// ---- graph.cu ---------------------------------------------------------------
void eval_partition(sphynx_graph *g, const int32_t *part, int K, double *cut, double *cut2,
                    double *imb);

}  // namespace sphynx
