/*
 * sphynx.h -- C ABI of the GB300 spectral graph partitioner.
 *
 * The library computes a K-way partition of an undirected graph the way the
 * Sphynx partitioner does (Acer, Boman, Glusa, Rajamanickam, "Sphynx: a
 * parallel multi-GPU graph partitioner for distributed-memory systems",
 * Algorithm 2): it forms a graph Laplacian, finds its d = floor(log2 K) + 1
 * smallest eigenvectors with preconditioned LOBPCG (Algorithm 1), drops the
 * first, and cuts the remaining d - 1 coordinates into K parts with
 * multi-jagged multisection (Sec. 4).  Every step runs in the library's own
 * CUDA kernels for sm_103a on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: every call returns int, 0 (SPHYNX_OK) on success or one of the
 *   SPHYNX_ERR_* codes below; nothing throws across the ABI.  After a
 *   failure, sphynx_last_error() gives a message (thread-local, valid until
 *   the next call on the same thread).
 * - Graph: CSR of a simple undirected graph with n vertices and nnz stored
 *   entries: row_ptr int64[n+1] (row_ptr[0] = 0, non-decreasing,
 *   row_ptr[n] = nnz), col int32[nnz] (column indices strictly increasing in
 *   each row, in [0, n), no self-loops), both (i,j) and (j,i) present.
 *   Optional edge weights float32[nnz] (positive, symmetric) and vertex
 *   weights int64[n] (>= 1).  NULL weights mean unit weights.
 * - Blocks of vectors are row-major n x ld arrays (ld >= ncols, element
 *   (i, j) at i*ld + j); "device" means a pointer to memory of the handle's
 *   GPU (e.g. from torch.empty(..., device="cuda")).
 * - Ownership: the caller owns every buffer it passes.  The handle owns its
 *   device copy of the graph and its workspaces; sphynx_destroy frees them.
 * - Streams: all work of a handle is ordered on the stream given to
 *   sphynx_create (a cudaStream_t, NULL = legacy default stream).  Calls that
 *   return results in host memory synchronise that stream before returning.
 *   A handle is not thread-safe; distinct handles may be used concurrently.
 */
#ifndef SPHYNX_H
#define SPHYNX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SPHYNX_OK 0
#define SPHYNX_ERR_INVALID_ARG 1   /* bad pointer, size, option or CSR structure */
#define SPHYNX_ERR_NOT_SYMMETRIC 2 /* some (i,j) has no matching (j,i) of equal weight */
#define SPHYNX_ERR_ISOLATED 3      /* a vertex has no edge (generalized/normalized need deg > 0) */
#define SPHYNX_ERR_OOM 4           /* device allocation failed */
#define SPHYNX_ERR_CUDA 5          /* a CUDA runtime call or kernel launch failed */
#define SPHYNX_ERR_NOCONV 6        /* LOBPCG hit max_iter; outputs hold the last iterate */
#define SPHYNX_ERR_BREAKDOWN 7     /* Rayleigh-Ritz basis lost rank beyond recovery */
#define SPHYNX_ERR_UNSUPPORTED 8   /* a size outside the documented limits */

/* ---- sphynx_create flags ------------------------------------------------ */
#define SPHYNX_HOST_PTRS 0u     /* row_ptr/col/weights are host pointers (copied) */
#define SPHYNX_DEVICE_PTRS 1u   /* they are device pointers (adopted: keep alive until destroy;
                                   col and edge_w 16-byte aligned, row_ptr and vtx_w 8-byte) */
#define SPHYNX_VALIDATE 2u      /* check CSR structure and symmetry on the GPU */

/* ---- option enums ------------------------------------------------------- */
/* Laplacian / eigenproblem (Sec. 3.2): L_C x = lambda x (Eq. 2),
 * L_C x = lambda D x, or L_N x = lambda x (Eq. 3). */
#define SPHYNX_COMBINATORIAL 0
#define SPHYNX_GENERALIZED 1
#define SPHYNX_NORMALIZED 2
/* Preconditioner (Sec. 5): none, Jacobi M = diag(L)^-1 (Sec. 5.1), the
 * GMRES polynomial p_k(L) (Sec. 5.2), or aggregation multigrid (Sec. 5.3,
 * parameters of Sec. 6.2.2): one symmetric V-cycle on L_C per application,
 * plain aggregation, degree-3 Chebyshev smoothing (eigenvalue ratio 7,
 * lambda_max from 10 power-iteration steps, 100 on the coarsest level), at
 * most 5 levels, and a Chebyshev coarse solve.  The multigrid preconditioner
 * approximates L_C^{-1}, so it takes the combinatorial and generalized
 * problems (INVALID_ARG with the normalized one) and single graphs
 * (UNSUPPORTED in sphynx_partition_batch). */
#define SPHYNX_PRECOND_NONE 0
#define SPHYNX_PRECOND_JACOBI 1
#define SPHYNX_PRECOND_POLY 2
#define SPHYNX_PRECOND_AMG 3
/* Arithmetic.  FP64: every block and product in double.  FP32: blocks in
 * float with float products; Gram matrices accumulated to double, the
 * Cholesky / Rayleigh-Ritz small problems and the residual norms in double.
 * MIXED_BF16: as FP32, but the polynomial preconditioner's chain vectors
 * are stored in bfloat16 (products still accumulate in float). */
#define SPHYNX_FP64 0
#define SPHYNX_FP32 1
#define SPHYNX_MIXED_BF16 2
/* Initial block (Sec. 6.2.1): seeded random, or piecewise constant. */
#define SPHYNX_INIT_RANDOM 0
#define SPHYNX_INIT_PIECEWISE 1
/* Element types of user blocks passed to the step-level calls. */
#define SPHYNX_DT_F64 0
#define SPHYNX_DT_F32 1
#define SPHYNX_DT_BF16 2
/* Convergence test of a Ritz pair (Sec. 6.3.2 names the tolerance, not the
 * test; x_i is B-normalised): REL_THETA ||r_i||_{B^-1} <= tol |theta_i|, or
 * ABS ||r_i||_{B^-1} <= tol.  Under both, the eigenvalue-zero vector is also
 * accepted at the rounding floor (|theta| <= 10 u rho and ||r|| <= 10 u rho
 * (max degree + 1), rho a Gershgorin bound of the operator). */
#define SPHYNX_CONV_REL_THETA 0
#define SPHYNX_CONV_ABS 1
/* sphynx_options.flags */
#define SPHYNX_OUT_DEVICE 1u    /* part_out of sphynx_partition is a device pointer */

/* Largest block size the kernels are built for: d = floor(log2 K) + 1 <= 16,
 * i.e. K < 65536. */
#define SPHYNX_MAX_NEV 16
/* Largest polynomial degree (Sec. 5.2 uses 25). */
#define SPHYNX_MAX_POLY_DEGREE 64
/* Roots the polynomial setup may add to keep p positive (sphynx_precond_setup):
 * up to 4 where p dips below zero, and one to make the count odd. */
#define SPHYNX_MAX_ADDED_ROOTS 5

typedef struct sphynx_graph *sphynx_handle;

typedef struct {
  int32_t laplacian;   /* SPHYNX_COMBINATORIAL | _GENERALIZED | _NORMALIZED   */
  int32_t precond;     /* SPHYNX_PRECOND_*                                     */
  int32_t poly_degree; /* k of p_k, 1..SPHYNX_MAX_POLY_DEGREE (default 25)     */
  int32_t precision;   /* SPHYNX_FP64 | SPHYNX_FP32 | SPHYNX_MIXED_BF16        */
  int32_t init;        /* SPHYNX_INIT_RANDOM | SPHYNX_INIT_PIECEWISE           */
  int32_t max_iter;    /* LOBPCG iteration cap (default 1000)                  */
  double tol;          /* LOBPCG tolerance (default 1e-3)                      */
  uint64_t seed;       /* seeds the random block and the polynomial start      */
  uint32_t flags;      /* SPHYNX_OUT_DEVICE                                    */
  int32_t sync_every;  /* iterations between host convergence checks (0=auto)  */
  int32_t stall_window;/* 0 (default): iterate until converged or max_iter.
                          w > 0: also stop, with NOCONV and the best iterate,
                          once every unconverged column has gone w iterations
                          without its residual falling below 0.9 x its best so
                          far, its best residual being under the noise floor
                          10 u rho (FP32 blocks cannot reach tol * theta when
                          that is below the FP32 rounding of L x)             */
  int32_t conv;        /* SPHYNX_CONV_REL_THETA (default) | SPHYNX_CONV_ABS     */
  int32_t refine_rounds;/* sphynx_partition: 0 (default) leaves the multi-jagged
                          partition as it is; r > 0 runs at most r rounds of
                          greedy refinement (sphynx_refine, eps = 0.01) on it  */
  int32_t reserved[3];
} sphynx_options;

typedef struct {
  int32_t status;        /* status of the LOBPCG solve (OK / NOCONV / BREAKDOWN)  */
  int32_t iterations;    /* LOBPCG iterations (Algorithm 1 loop trips)            */
  int32_t nev;           /* d                                                     */
  int32_t svqb_steps;    /* Rayleigh-Ritz steps that fell back from Cholesky       */
  double eigenvalues[SPHYNX_MAX_NEV]; /* Ritz values, ascending                    */
  double resnorm[SPHYNX_MAX_NEV];     /* ||L x - theta B x||_{B^-1} per column     */
  double ms_total;       /* wall time of the call (host clock)                     */
  double ms_setup;       /* preconditioner setup (device events)                   */
  double ms_lobpcg;      /* eigensolve incl. setup (device events)                 */
  double ms_mj;          /* embedding + multi-jagged (device events)               */
  double ms_eval;        /* cut and imbalance (device events)                      */
  double ms_spmm;        /* summed duration of the Laplacian SpMM launches         */
  int64_t spmm_launches; /* Laplacian SpMM launches                                 */
  double spmm_bytes;     /* algorithmic bytes of those launches                    */
  int64_t kernel_launches; /* all kernels this call launched                      */
  double cut;            /* Eq. 1                                                  */
  double cut_twice;      /* Eq. 1 counted from both endpoints (the paper's tables) */
  double imbalance;      /* max_k W_k / W_avg                                      */
  /* the three SpMM figures above split by the precision of the input block,
     indexed by SPHYNX_DT_F64, _F32, _BF16 (the BF16 entries are the
     polynomial-chain steps of SPHYNX_MIXED_BF16)                               */
  double ms_spmm_by_dt[3];
  double spmm_bytes_by_dt[3];
  int64_t spmm_launches_by_dt[3];
  int32_t fp64_finished; /* sphynx_partition_batch with float blocks: graphs that
                            stalled at the float rounding floor above tol |theta|
                            and finished in FP64 blocks from their float iterate */
  int32_t refine_moves;  /* vertices moved by greedy refinement (refine_rounds)  */
  double ms_phase[2];    /* sphynx_partition_batch: wall time of the eigensolve in
                            the requested precision and of the FP64 finishing
                            (0 when no graph was promoted)                      */
  int32_t loop_iters[2]; /* sphynx_partition_batch: LOBPCG iterations each phase's
                            captured loop ran (the most any graph of it took)   */
} sphynx_stats;

typedef struct {
  int64_t n, nnz;
  int64_t max_degree;        /* largest number of neighbours                       */
  double max_wdegree;        /* largest weighted degree                            */
  int64_t total_vweight;     /* sum of vertex weights                              */
  int64_t long_rows;         /* rows the SpMM routes to the long-row kernel        */
  int32_t weighted;          /* edge weights present                               */
  int32_t spmm_variant;      /* short-row schedule the autotuner chose at create
                                from a float 8-column product and uses for every
                                product: 0 = CSR staged in shared memory,
                                1 = SELL-32, 2 = SELL-32 with shared-pattern slices */
  float tuned_us_csr;        /* the two schedules' times for that product (us)    */
  float tuned_us_sell;
  int64_t sell_slices;       /* SELL-32 slices (32 rows each)                      */
  int64_t sell_narrow_slices;/* slices whose entries all lie within 32767 of their
                                row, stored as 16-bit offsets instead of 32-bit
                                column indices                                      */
  double spmm_graph_bytes;   /* bytes of graph structure one product reads with the
                                chosen schedule (indices, weights, row metadata)   */
  int32_t regular;           /* 1 if max degree <= 10 x average degree (Sec. 6.1)  */
  int32_t spmm_med_max;      /* the autotuner's choice: rows with 33 to this many
                                neighbours use the medium-row kernel (a group of
                                lanes per row), longer rows the long-row kernels
                                (a warp per 1024-entry piece); 32 means none are
                                medium                                              */
  int32_t sell_stride;       /* the autotuner's SELL-32 slice order: the four warps
                                of a block take slices this many apart (1, 2, 4, 8
                                or 16), so that on a mesh a block's rows can lie
                                on neighbouring grid lines and share gathered rows
                                of X in L1                                          */
  float tuned_us_pattern;    /* the shared-pattern schedule's time (0: not built)  */
  int64_t sell_pattern_slices;/* slices whose 32 rows' offsets col - row take at
                                most 31 distinct 16-bit values (unweighted graphs):
                                the shared-pattern schedule (spmm_variant 2) stores
                                that union once per slice plus a 32-bit entry mask
                                per row instead of one offset per entry           */
} sphynx_graph_info;

/* Fill *opt with the defaults listed in sphynx_options. */
void sphynx_default_options(sphynx_options *opt);

/* Fill *opt with Sphynx's defaults for this graph and preconditioner
 * (Sec. 6.3.1, decision flow of Fig. 2): the graph is regular when its
 * largest degree is at most 10 times its average degree (Sec. 6.1; compared
 * exactly as max_degree * n <= 10 * nnz).  Regular graphs get the
 * combinatorial problem, tol 1e-3 and the random start; irregular graphs get
 * the generalized problem (Jacobi or no preconditioner) or the normalized one
 * (polynomial), tol 1e-2 and the piecewise-constant start (Sec. 6.2.1).
 * precond: SPHYNX_PRECOND_*.  Other fields as sphynx_default_options.
 * Errors: INVALID_ARG. */
int sphynx_default_options_for(sphynx_handle g, int32_t precond, sphynx_options *opt);

/* Message of the last failed call on this thread ("" if none). */
const char *sphynx_last_error(void);

/* Create a graph handle (Sec. 3.1: G with vertex weights and edge costs).
 * Copies (HOST_PTRS) or adopts (DEVICE_PTRS) the CSR, computes weighted
 * degrees, D^{-1/2} and the SpMM plan, and with SPHYNX_VALIDATE checks the
 * structure and symmetry on the GPU.  `stream` is a cudaStream_t.
 * Errors: INVALID_ARG, NOT_SYMMETRIC, OOM, CUDA, UNSUPPORTED (n >= 2^31,
 * nnz >= 2^40, or total vertex weight times 2^22 overflowing int64). */
int sphynx_create(const int64_t *row_ptr, const int32_t *col, const float *edge_w,
                  const int64_t *vtx_w, int64_t n, int64_t nnz, uint32_t flags,
                  void *stream, sphynx_handle *out);

/* Release the handle and its device memory (NULL is ignored). */
void sphynx_destroy(sphynx_handle g);

/* Sizes and degree statistics of the graph (host struct). */
int sphynx_get_info(sphynx_handle g, sphynx_graph_info *info);

/* Pin the short-row SpMM schedule of the handle: 0 = CSR staged in shared
 * memory, 1 = SELL-32, 2 = SELL-32 with shared-pattern slices (only when the
 * graph has such slices, see sphynx_graph_info), -1 = time them again and keep
 * the fastest (what sphynx_create does).  All give the same products up to
 * rounding order; 1 and 2 sum every row in the same order.
 * Errors: INVALID_ARG. */
int sphynx_set_spmm_variant(sphynx_handle g, int32_t variant);

/* Override the autotuner's medium-row ceiling: rows with 33 to med_max
 * neighbours use the medium-row kernel, longer rows the long-row kernels
 * (med_max in [32, 4096]; 32: no medium rows).  Rebuilds the handle's plan
 * (reads row_ptr back from the device).  For tests and profiling.
 * Errors: INVALID_ARG. */
int sphynx_set_spmm_med_max(sphynx_handle g, int32_t med_max);

/* Override the autotuner's SELL-32 slice order: the four warps of a block take
 * slices `stride` rows-of-32 apart (1, 2, 4, 8 or 16), or -1 to time every
 * stride on a float 8-column product again and keep the fastest (what
 * sphynx_create does when it picks SELL-32).  The order changes which block
 * computes a row, never the row's value.  For tests and profiling.
 * Errors: INVALID_ARG, OOM (-1 allocates two n x 8 float blocks while it runs). */
int sphynx_set_spmm_sell_stride(sphynx_handle g, int32_t stride);

/* Weighted degrees deg(v_i) (Sec. 3.2: the diagonal of L_C) into a device
 * double[n]. */
int sphynx_degrees(sphynx_handle g, double *deg_out);

/* Y = L X for the chosen Laplacian without forming L (Eqs. 2-3 and the
 * weighted rule of Sec. 3.2; the generalized problem's operator is L_C).
 * X: device n x ldx block of dtype SPHYNX_DT_*; Y: device n x ldy block of
 * double (F64 input) or float (F32/BF16 input).  ncols <= 16.  Padding
 * columns of Y (ncols..ldy) are not written. */
int sphynx_laplacian_apply(sphynx_handle g, int32_t laplacian, int32_t dtype, const void *x,
                           int32_t ldx, void *y, int32_t ldy, int32_t ncols);

/* One step of the polynomial preconditioner's product form (Sec. 5.2), the
 * fused kernel every application of the polynomial runs k - 1 times: with t
 * the input block and L the operator of `laplacian` (L_C for the generalized
 * problem),
 *   t_out = t - (L t) / theta_cur
 * and the accumulator y of p(L) t gathers the step's terms:
 *   yterms 2: y = (first ? 0 : y) + t / theta_cur + t_out / theta_next
 *   yterms 1: y = y + t_out / theta_next
 *   yterms 0: y unchanged.
 * The terms use the stored (rounded) t_out.  t, t_out: device n x ld blocks
 * (ld = round4(ncols), rows exactly ld apart) of dtype_in / dtype_out: F64 ->
 * F64, F32 -> F32 or BF16, BF16 -> BF16; y: device n x ld block of double (F64)
 * or float.  Float and bfloat16 steps multiply by the float-rounded
 * reciprocals of the roots and accumulate in float.  first = 1 needs
 * yterms = 2.  Asynchronous on the handle's stream; the reciprocals are
 * uploaded only when the roots differ from the previous call's.  Errors:
 * INVALID_ARG, ISOLATED. */
int sphynx_poly_step(sphynx_handle g, int32_t laplacian, int32_t dtype_in, const void *t, int32_t dtype_out,
                     void *t_out, void *y, int32_t ld, int32_t ncols, double theta_cur, double theta_next,
                     int32_t yterms, int32_t first);

/* Set up the preconditioner of `opt` (Sec. 5) and, for the polynomial,
 * return its roots in application order in host
 * double[poly_degree + SPHYNX_MAX_ADDED_ROOTS] (may be NULL): the harmonic
 * Ritz values of k = poly_degree Lanczos steps, plus a second copy of a root
 * for each time p was not positive on a grid over (0, largest root] (at most
 * 4), plus a copy of the largest root if the count is then even (p is then
 * positive above the largest root too; LOBPCG needs a positive definite
 * preconditioner), Leja ordered; the entries after the last root are +inf.  For multigrid, build the level hierarchy for opt->seed
 * (kept by the handle and reused while the seed is the same); a coarse row
 * sorts its entries in shared memory when its aggregate's rows hold at most
 * 8192 of them and in global scratch (chunks of at most 512 MiB) otherwise;
 * errors: UNSUPPORTED when an aggregate's rows hold 2^31 or more entries.
 * Jacobi and none need no setup. */
int sphynx_precond_setup(sphynx_handle g, const sphynx_options *opt, double *roots_out);

/* H = M R for the preconditioner set up by the last sphynx_precond_setup
 * (or Jacobi/none from `opt`).  R, H: device n x ld blocks of float (FP32 /
 * MIXED_BF16 precision) or double (FP64); ncols <= 16. */
int sphynx_precond_apply(sphynx_handle g, const sphynx_options *opt, const void *r, void *h,
                         int32_t ld, int32_t ncols);

/* One level of the multigrid hierarchy built by sphynx_precond_setup (or by
 * a partition with SPHYNX_PRECOND_AMG): level 0 is the graph itself, level
 * l + 1 the aggregate graph of level l, whose edge (I, J) weighs the sum of
 * the weights of level l's edges between aggregates I and J, so that its
 * combinatorial Laplacian is the Galerkin product P^T L_C P (Sec. 5.3).
 * info (host, may be NULL) receives the level count, the level's size, its
 * aggregate count (0 on the coarsest level) and its Chebyshev lambda_max.
 * The device outputs may be NULL: agg_out int32[n] (the aggregate of each
 * vertex; INVALID_ARG on the coarsest level), row_ptr_out int64[n + 1],
 * col_out int32[nnz] (sorted within each row), w_out float[nnz] (levels >= 1).
 * Errors: INVALID_ARG (no hierarchy, level out of range). */
typedef struct {
  int32_t levels;      /* levels in the hierarchy                        */
  int32_t reserved;
  int64_t n, nnz;      /* this level's vertices and stored entries       */
  int64_t n_next;      /* aggregates (vertices of the next level), 0 on the coarsest */
  double lambda_max;   /* Chebyshev interval top: min(1.1 x power estimate, 2) */
} sphynx_amg_level_info;
int sphynx_amg_level(sphynx_handle g, int32_t level, sphynx_amg_level_info *info, int32_t *agg_out,
                     int64_t *row_ptr_out, int32_t *col_out, float *w_out);

/* Gram matrices of Rayleigh-Ritz (Sec. 3.3, the Rayleigh-Ritz step of Algorithm 1):
 * G_A = S^T (L S) and G_B = S^T B S, where S = [S_0 | S_1 | S_2] and
 * LS = [LS_0 | LS_1 | LS_2] are given as nblk (1..3) device n x ld blocks of
 * dtype F32 or F64 (each ld columns wide, 4 | ld, ld <= 16), and B is
 * diag(bdiag) (device double[n]) or the identity (bdiag = NULL).  Outputs
 * are host double[(nblk*ld)^2], row-major and symmetric: both matrices are
 * formed from their upper triangles (S^T L S is symmetric when LS = L S).
 * Accumulation: products in the input type, short sums in the input type,
 * then a (hi, lo) float pair (float input) or double, per-CTA partials in
 * double added in a fixed order.
 * Scratch: allocated per call with cudaMallocAsync on `stream`. */
int sphynx_gram(int32_t dtype, const void *const *s_blocks, const void *const *ls_blocks,
                int32_t nblk, int32_t ld, int64_t n, const double *bdiag, double *ga_out,
                double *gb_out, void *stream);

/* Rayleigh-Ritz on the GPU in FP64 (Sec. 3.3): given host G_A, G_B (m x m,
 * m <= 48) and an active mask (host int32[m], nonzero = column in S),
 * returns the nev smallest Ritz values (host double[nev]) and coefficients
 * Y (host double[m * nev], row-major m x nev, zero rows for inactive
 * columns).  u_work sets the rank threshold 10 m u_work.  *used_svqb tells
 * whether the Cholesky factor was replaced by an eigendecomposition. */
int sphynx_rayleigh_ritz(const double *ga, const double *gb, const int32_t *active, int32_t m,
                         int32_t nev, double u_work, double *theta_out, double *y_out,
                         int32_t *used_svqb, void *stream);

/* LOBPCG (Algorithm 1) for the nev smallest eigenpairs of the problem of
 * `opt`.  x0: optional host double[n * nev] initial block (NULL = the
 * seeded block of opt->init).  x_out: device n x ldx block of double (FP64)
 * or float (FP32/MIXED_BF16) with the B-orthonormal Ritz vectors;
 * theta_out / resnorm_out: host double[nev] (may be NULL).
 * Returns OK, NOCONV or BREAKDOWN (outputs valid for the last two). */
int sphynx_eigensolve(sphynx_handle g, const sphynx_options *opt, int32_t nev, const double *x0,
                      void *x_out, int32_t ldx, double *theta_out, double *resnorm_out,
                      sphynx_stats *stats);

/* Multi-jagged multisection (Sec. 4) of n points with `dims` coordinates
 * (device n x ldc block of SPHYNX_DT_F64 or _F32), vertex weights (device
 * int64[n] or NULL = unit) into K parts: each section owning k parts splits
 * ceil(k/2) | floor(k/2) along dimension (level mod dims) at the prefix of
 * the (coordinate, vertex id) order minimising |k W_left - ceil(k/2) W|,
 * ties to the shorter prefix (-0 == +0; NaN is INVALID_ARG).
 * part_out: device int32[n].  Scratch is allocated per call.  Bit-exact. */
int sphynx_mj(int32_t dtype, const void *coords, int32_t ldc, int32_t dims, int64_t n,
              const int64_t *vtx_w, int32_t K, int32_t *part_out, void *stream);

/* sphynx_mj without any device allocation (the paper has no counterpart).
 * It serves callers that cannot let a library allocate device memory: a
 * framework whose own caching allocator has already reserved the device's
 * memory, or an application that budgets all device memory at start-up and
 * allows no allocation afterwards.  Same arguments and the same bit-exact
 * result as sphynx_mj; part_out and every input stay caller-owned.  Scratch
 * lives in a fixed 16 MiB array in device memory that every GPU loading the
 * library holds until the process exits; calls needing more (roughly
 * 8 n + 5200 K bytes; n <= 2^20 with K <= 1024 fits) fail with
 * SPHYNX_ERR_UNSUPPORTED, as K > 2^20 does in both entry points.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and should therefore come before any stream
 * capture.  Like sphynx_mj, every call reads two values back to the host (a
 * NaN / vertex-weight flag and the total vertex weight), so it synchronises
 * `stream` twice, and it uploads its section tables from pageable host
 * memory.  All calls share the one array and each call clears what it needs
 * cleared: calls whose GPU work overlaps (different streams, or concurrent
 * host threads) race and must be serialised by the caller. */
int sphynx_mj_noalloc(int32_t dtype, const void *coords, int32_t ldc, int32_t dims, int64_t n,
                      const int64_t *vtx_w, int32_t K, int32_t *part_out, void *stream);

/* Cutsize (Eq. 1, exact: integer for unit weights, exact fixed point for
 * float weights, rounded once) and imbalance max_k W_k / W_avg (Sec. 3.1)
 * of a partition given as device int32[n] with values in [0, K). */
int sphynx_eval(sphynx_handle g, const int32_t *part, int32_t K, double *cut,
                double *cut_twice, double *imbalance);

/* Algorithm 2: K-way partition.  part_out: int32[n], host memory unless
 * opt->flags has SPHYNX_OUT_DEVICE.  cut_out / imbalance_out / stats may be
 * NULL.  Every call sets up its preconditioner anew (the polynomial's roots,
 * the multigrid hierarchy), and stats->ms_setup times that setup.  Returns
 * OK, or NOCONV / BREAKDOWN with a valid partition of the last iterate;
 * INVALID_ARG for bad options (among them the multigrid preconditioner with
 * the normalized problem). */
int sphynx_partition(sphynx_handle g, int32_t K, const sphynx_options *opt, int32_t *part_out,
                     double *cut_out, double *imbalance_out, sphynx_stats *stats);

/* Greedy refinement of a K-way partition (Sec. 7 proposes a greedy
 * improvement step after the spectral partition; the paper gives no
 * algorithm, this is the library's parallel reading).  part: device
 * int32[n] with values in [0, K), changed in place.  Each round: every
 * vertex of at most 256 neighbours finds the external part it is most
 * connected to (the smallest part on ties) and its gain, that connection
 * minus its connection to its own part, in exact integers (edge weights
 * w * 2^s as the exact cut sums them, integer vertex weights); a vertex of
 * positive gain is selected when no neighbour of positive gain outranks it
 * (higher gain, or equal gain and a lower id), so the selected vertices are
 * pairwise non-adjacent and each gain is exactly the cut its move removes;
 * a part takes all the selected vertices aimed at it when its weight stays
 * within cap = floor((1 + eps) W_total / K) (evaluated in double), otherwise
 * only the one of highest priority if that fits.  Rounds stop when none
 * moves or after max_rounds.  The cut never rises and no part grows beyond
 * max(cap, its weight before).  Deterministic and bit-exact.  cut_out,
 * imbalance_out (as sphynx_eval), moves_out, rounds_out: host, may be NULL.
 * Errors: INVALID_ARG (a part id outside [0, K), eps < 0), UNSUPPORTED
 * (batch handles; weights too wide for exact integer gains). */
int sphynx_refine(sphynx_handle g, int32_t *part, int32_t K, double eps, int32_t max_rounds, double *cut_out,
                  double *imbalance_out, int32_t *moves_out, int32_t *rounds_out);

/* A batch of graphs in one handle, for partitioning thousands of graphs of
 * uneven sizes in one call (Algorithm 2 applied to every graph; the paper
 * has no batched form).  The graphs come as one block-diagonal CSR over
 * n = all vertices: graph q owns vertices [graph_ptr[q], graph_ptr[q+1]) and
 * every edge of a graph stays inside that range (checked: INVALID_ARG).
 * graph_ptr: host int64[count + 1], graph_ptr[0] = 0, graph_ptr[count] = n,
 * every graph non-empty.  The other arguments, ownership and errors are
 * those of sphynx_create.  With host arrays (SPHYNX_HOST_PTRS) the handle
 * stores every graph's vertices in reverse Cuthill-McKee order (computed on
 * the host's cores, within each graph), so that a row's neighbours lie near
 * it and the products' gathers share cache lines; sphynx_partition_batch
 * takes and returns everything in the caller's numbering, and draws the
 * same random numbers per vertex as an unordered batch.  With device arrays
 * the caller's order is kept.  The handle also serves the single-step
 * calls, which see the block-diagonal graph in the handle's row order. */
int sphynx_create_batch(const int64_t *row_ptr, const int32_t *col, const float *edge_w,
                        const int64_t *vtx_w, const int64_t *graph_ptr, int32_t count, int64_t n,
                        int64_t nnz, uint32_t flags, void *stream, sphynx_handle *out);

/* Partition every graph of a batch handle into K parts: each graph gets its
 * own LOBPCG (Algorithm 1: its own Ritz values, convergence test and soft
 * locking), embedding and multi-jagged partition, as a single-graph call
 * with the same options would; its random initial block is the one that call
 * would draw.  The LOBPCG iterations of all graphs run as one CUDA graph
 * launch whose conditional loop repeats on the device until every graph has
 * converged or reached max_iter; a converged graph drops out (after every
 * convergence test the device rebuilds the lists of row blocks and chunks
 * that hold graphs still iterating, and every product and reduction of the
 * next iteration walks those lists with a fixed grid).  Jacobi, the
 * polynomial (degree >= 2: every graph's own roots from its own Lanczos
 * steps, Sec. 5.2, applied with one chain over all graphs) or no
 * preconditioner; random initial block.
 * part_out: int32[n] part ids local to each graph (0..K-1), host memory
 * unless opt->flags has SPHYNX_OUT_DEVICE.  cuts, imbalances (double[count]),
 * eigenvalues (double[count * d], d = floor(log2 K) + 1, each graph's Ritz
 * values ascending), iterations and status (int32[count], OK or NOCONV per
 * graph): host arrays, each may be NULL.  stats (may be NULL): status OK only if every graph
 * converged, iterations = the largest, fp64_finished = graphs that went on in
 * FP64 blocks.  With float blocks (FP32, MIXED_BF16) a graph whose tol |theta|
 * lies below the float rounding floor of its residual stops in float once an
 * unconverged column whose target is below u rho (rho the Gershgorin bound of
 * the noise floor) has a residual within 10 u rho, or once every unconverged
 * column has gone stall_window iterations (20 when 0) without a 10 % gain at
 * that floor; the graph then resumes in FP64 blocks from its float iterate (iterations count on, under the same max_iter), and the
 * embedding and multi-jagged step then run on double coordinates for all
 * graphs.  Errors: INVALID_ARG (not a batch
 * handle), UNSUPPORTED (multigrid preconditioner, polynomial of degree 1,
 * piecewise start, K x count > 2^20), BREAKDOWN (a graph's polynomial setup
 * failed), CUDA, OOM. */
int sphynx_partition_batch(sphynx_handle g, int32_t K, const sphynx_options *opt, int32_t *part_out,
                           double *cuts, double *imbalances, double *eigenvalues, int32_t *iterations,
                           int32_t *status, sphynx_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* SPHYNX_H */
