// lobpcg.cu -- host orchestration of the hot path: preconditioner setup
// (Sec. 5), LOBPCG (Algorithm 1), the embedding and multi-jagged step and the
// partition metrics (Algorithm 2).
//
// All iteration state lives on the GPU.  One LOBPCG iteration is a fixed
// sequence of launches on the handle's stream:
//   [polynomial chain: k-1 fused SpMM steps,
//    or one multigrid V-cycle]                H = M R
//   SpMM                                       LH = L H
//   Gram + fixed-order reduction               G_A = S^T L S, G_B = S^T B S, S = [X H P]
//   Rayleigh-Ritz (one CTA, FP64)              Y, Theta
//   update                                     X' = S Y, P' = [0 H P] Y, LP' = [0 LH LP] Y
//   SpMM                                       LX' = L X'
//   residual (+ Jacobi)                        R = LX' - B X' Theta, norms
//   convergence test                           conv, done
// Every launch is skipped on the device once `done` is set, so the host only
// polls the flag every few iterations.
#include "internal.cuh"

#include <chrono>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

namespace sphynx {

namespace {

int round4(int b) { return (b + 3) & ~3; }

DT block_dt(int precision) { return precision == SPHYNX_FP64 ? DT::F64 : DT::F32; }
DT chain_dt(int precision) {
  return precision == SPHYNX_FP64 ? DT::F64 : (precision == SPHYNX_MIXED_BF16 ? DT::BF16 : DT::F32);
}
int op_of(int laplacian) { return laplacian == SPHYNX_NORMALIZED ? SPHYNX_NORMALIZED : SPHYNX_COMBINATORIAL; }

void check_options(const sphynx_graph *g, const sphynx_options *o) {
  if (!o) fail(SPHYNX_ERR_INVALID_ARG, "options are NULL");
  if (o->laplacian < 0 || o->laplacian > 2) fail(SPHYNX_ERR_INVALID_ARG, "laplacian %d", o->laplacian);
  if (o->precond < 0 || o->precond > 3) fail(SPHYNX_ERR_INVALID_ARG, "precond %d", o->precond);
  if (o->precond == SPHYNX_PRECOND_AMG && o->laplacian == SPHYNX_NORMALIZED)
    fail(SPHYNX_ERR_INVALID_ARG, "the multigrid preconditioner approximates L_C^{-1}: combinatorial or generalized "
         "problem only");
  if (o->precision < 0 || o->precision > 2) fail(SPHYNX_ERR_INVALID_ARG, "precision %d", o->precision);
  if (o->init < 0 || o->init > 1) fail(SPHYNX_ERR_INVALID_ARG, "init %d", o->init);
  if (o->precond == SPHYNX_PRECOND_POLY && (o->poly_degree < 1 || o->poly_degree > SPHYNX_MAX_POLY_DEGREE))
    fail(SPHYNX_ERR_INVALID_ARG, "poly_degree %d", o->poly_degree);
  if (o->max_iter < 0) fail(SPHYNX_ERR_INVALID_ARG, "max_iter < 0");
  if (o->stall_window < 0) fail(SPHYNX_ERR_INVALID_ARG, "stall_window < 0");
  if (o->conv != SPHYNX_CONV_REL_THETA && o->conv != SPHYNX_CONV_ABS) fail(SPHYNX_ERR_INVALID_ARG, "conv %d", o->conv);
  if (o->refine_rounds < 0) fail(SPHYNX_ERR_INVALID_ARG, "refine_rounds < 0");
  if (!(o->tol >= 0.0)) fail(SPHYNX_ERR_INVALID_ARG, "tol");
  if (o->laplacian != SPHYNX_COMBINATORIAL && g->isolated > 0)
    fail(SPHYNX_ERR_ISOLATED, "%lld vertices without edges: the %s problem needs deg > 0",
         static_cast<long long>(g->isolated), o->laplacian == SPHYNX_NORMALIZED ? "normalized" : "generalized");
}

void plain_spmm(sphynx_graph *g, int lap_op, DT dt, const void *x, void *y, int ld, int b, const int *done) {
  SpmmArgs a{};
  a.lap = lap_op;
  a.tin = dt;
  a.ld_x = ld;
  a.ld_y = ld;
  a.bp = ld;
  a.b_true = b;
  a.x = x;
  a.y = y;
  a.mode = 0;
  a.done = done;
  spmm(g, a);
}

// ---- polynomial preconditioner (Sec. 5.2) ----------------------------------
void poly_setup(sphynx_graph *g, const sphynx_options *o) {
  const int k = o->poly_degree;
  const DT dt = block_dt(o->precision);
  const size_t es = dt_size(dt);
  const int lap = op_of(o->laplacian);
  const int64_t n = g->n;
  const int64_t ldv = (n + 3) & ~static_cast<int64_t>(3);   // column-major basis, 16-byte aligned columns
  cudaStream_t st = g->stream;
  // column 0 holds the normalised null vector of L and column j + 1 the
  // Lanczos vector v_j: both Gram-Schmidt passes orthogonalise against the null
  // vector too, which changes nothing in exact arithmetic but stops rounding
  // in a float basis from re-growing the null component over the k steps
  void *V = g->workspace("lz_V", static_cast<size_t>(ldv) * (k + 1) * es, false);
  void *v = g->workspace("lz_v", static_cast<size_t>(ldv) * es, false);
  void *w = g->workspace("lz_w", static_cast<size_t>(ldv) * es, false);
  const int grid = vec_grid(n);
  double *part = static_cast<double *>(g->workspace("lz_part", static_cast<size_t>(grid) * (SPHYNX_MAX_POLY_DEGREE + 2) * 8, false));
  double *small = static_cast<double *>(g->workspace("lz_small", 8 * (4 * SPHYNX_MAX_POLY_DEGREE + 16), true));
  double *alpha = small, *beta2 = small + SPHYNX_MAX_POLY_DEGREE, *h = small + 2 * SPHYNX_MAX_POLY_DEGREE;
  double *scal = small + 3 * SPHYNX_MAX_POLY_DEGREE + 2, *nrm = scal + 4;
  const int kcap = k + SPHYNX_MAX_ADDED_ROOTS;
  g->poly_inv.alloc((kcap + 1) * sizeof(double));
  g->poly_invf.alloc((kcap + 1) * sizeof(float));
  DevBuf roots, err;
  roots.alloc(kcap * sizeof(double));
  err.alloc(2 * sizeof(int));   // error flag, root count
  SPX_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int), st));

  launch_poly_start(st, dt, v, n, o->seed);
  launch_project_null(st, dt, v, n, lap, g->deg.as<double>(), part, grid, scal);
  launch_null_column(st, dt, V, n, lap, g->deg.as<double>(), scal);
  // beta_0^2 = ||v||^2, then v <- v / beta_0 and V[:, 1] = v
  launch_lanczos_dots(st, dt, v, ldv, 1, v, n, part, grid);
  launch_reduce_cols(st, part, grid, 1, nrm);
  launch_lanczos_next(st, dt, v, v, V, ldv, 1, n, nrm);
  g->ctr.launches += 8;
  for (int j = 0; j < k; ++j) {
    plain_spmm(g, lap, dt, v, w, 1, 1, nullptr);                 // w = L v_j
    for (int pass = 0; pass < 2; ++pass) {                       // two Gram-Schmidt passes
      launch_lanczos_dots(st, dt, V, ldv, j + 2, w, n, part, grid);
      launch_reduce_cols(st, part, grid, j + 2, h);
      if (pass == 0) SPX_CUDA(cudaMemcpyAsync(alpha + j, h + j + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
      launch_lanczos_sub(st, dt, V, ldv, j + 2, w, n, h, part, grid);
    }
    launch_reduce_cols(st, part, grid, 1, beta2 + j);            // beta_j^2 = ||w||^2
    if (j + 1 < k) launch_lanczos_next(st, dt, w, v, V, ldv, j + 2, n, beta2 + j);
    g->ctr.launches += 8;
  }
  launch_harmonic_ritz(st, alpha, beta2, k, roots.as<double>(), g->poly_inv.as<double>(), g->poly_invf.as<float>(),
                       err.as<int>(), err.as<int>() + 1);
  g->ctr.launches += 3;
  int herr[2] = {0, 0};
  g->poly_roots.assign(kcap, 0.0);
  SPX_CUDA(cudaMemcpyAsync(g->poly_roots.data(), roots.p, kcap * sizeof(double), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaMemcpyAsync(herr, err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  if (herr[0]) fail(SPHYNX_ERR_BREAKDOWN, "polynomial setup: Lanczos tridiagonal not positive definite (%d)", herr[0]);
  g->poly_roots.resize(herr[1]);
  g->poly_k = herr[1];
  g->poly_degree = k;
  g->poly_laplacian = lap;
}

// H = p(L) R in product form; R and H are n x ld blocks of the block type
void poly_apply(sphynx_graph *g, int precision, const void *r, void *h, int ld, int b, const int *done,
                bool r_bf16 = false) {
  const int k = g->poly_k;
  const DT dt = block_dt(precision), ct = chain_dt(precision);
  if (k == 1) {
    launch_poly_single(g->stream, dt, r, h, g->n, ld, g->poly_inv.as<double>(), done);
    g->ctr.launches++;
    return;
  }
  const size_t cs = dt_size(ct);
  void *c0 = g->workspace("chain0", static_cast<size_t>(g->n) * ld * cs, false);
  void *c1 = g->workspace("chain1", static_cast<size_t>(g->n) * ld * cs, false);
  void *ch[2] = {c0, c1};
  for (int i = 0; i + 1 < k; ++i) {
    SpmmArgs a{};
    a.lap = g->poly_laplacian;
    a.tin = i == 0 ? (r_bf16 ? DT::BF16 : dt) : ct;
    a.ld_x = ld;
    a.ld_y = ld;
    a.bp = ld;
    a.b_true = b;
    a.x = i == 0 ? r : ch[(i - 1) & 1];
    a.mode = 1;
    a.t_out = ch[i & 1];
    a.tout = ct;
    a.yacc = h;
    a.first = i == 0 ? 1 : 0;
    // y gathers two terms on even steps; an odd step leaves y alone unless
    // it is the last, which adds its output
    a.yterms = (i % 2 == 0) ? 2 : (i + 2 == k ? 1 : 0);
    a.inv = g->poly_inv.as<double>();
    a.invf = g->poly_invf.as<float>();
    a.i_cur = i;
    a.done = done;
    spmm(g, a);
  }
}

// ---- embedding: canonical rotation within clusters of equal Ritz values -------
// Eigenvectors of (nearly) equal eigenvalues are fixed only up to a rotation of
// their span, and the multi-jagged cuts depend on that rotation.  Within each
// run of Ritz values whose neighbours differ by at most tol (relative to the
// larger; the eigenvalue-zero column excluded) the columns E_c become E_c Q,
// Q the orthogonal polar factor of E_c^T Z_c with Z a seeded reference block
// (the orthogonal Procrustes rotation towards Z), so that the embedding
// depends on the span only.  Q = M (M^T M)^{-1/2}, from a cyclic Jacobi
// eigendecomposition of M^T M on the host (c is at most 16).
namespace {

void sym_eig_host(std::vector<double> &a, int c, std::vector<double> &v) {
  v.assign(static_cast<size_t>(c) * c, 0.0);
  for (int i = 0; i < c; ++i) v[i * c + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        tot += a[i * c + j] * a[i * c + j];
        if (i != j) off += a[i * c + j] * a[i * c + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < c; ++p)
      for (int q = p + 1; q < c; ++q) {
        const double apq = a[p * c + q];
        if (apq == 0.0) continue;
        const double tau = (a[q * c + q] - a[p * c + p]) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < c; ++k) {   // A <- A J (columns p, q)
          const double akp = a[k * c + p], akq = a[k * c + q];
          a[k * c + p] = cs * akp - sn * akq;
          a[k * c + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < c; ++k) {   // A <- J^T A (rows p, q)
          const double apk = a[p * c + k], aqk = a[q * c + k];
          a[p * c + k] = cs * apk - sn * aqk;
          a[q * c + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < c; ++k) {   // V <- V J
          const double vkp = v[k * c + p], vkq = v[k * c + q];
          v[k * c + p] = cs * vkp - sn * vkq;
          v[k * c + q] = sn * vkp + cs * vkq;
        }
      }
  }
}

}  // namespace

// ---- LOBPCG -------------------------------------------------------------------
struct EigenResult {
  int status = SPHYNX_OK;
  int iterations = 0;
  int svqb = 0;
  double theta[SPHYNX_MAX_NEV] = {0};
  double res[SPHYNX_MAX_NEV] = {0};
  const void *x = nullptr;   // final Ritz vectors (workspace)
  DT dt = DT::F64;
  int ld = 0;
  float ms_setup = 0;
};

EigenResult lobpcg(sphynx_graph *g, const sphynx_options *o, int b, const double *x0_host) {
  check_options(g, o);
  if (b < 1 || b > SPHYNX_MAX_NEV) fail(SPHYNX_ERR_UNSUPPORTED, "nev %d outside [1, %d]", b, SPHYNX_MAX_NEV);
  cudaStream_t st = g->stream;
  const int64_t n = g->n;
  const DT dt = block_dt(o->precision);
  const size_t es = dt_size(dt);
  const int ld = round4(b);
  const int lap = op_of(o->laplacian);
  const bool gen = o->laplacian == SPHYNX_GENERALIZED;
  const double u_work = o->precision == SPHYNX_FP64 ? 0x1.0p-53 : 0x1.0p-24;
  const double rho = lap == SPHYNX_COMBINATORIAL && !gen ? 2.0 * g->max_wdeg : 2.0;
  // noise floors of the eigenvalue-zero vector: |theta| within 10 u rho, and
  // ||r|| within the rounding bound of one row of L x, 10 u rho (d_max + 1)
  const double floor_th = 10.0 * u_work * rho;
  const double floor_res = floor_th * static_cast<double>(g->max_degree + 1);
  const size_t blk = static_cast<size_t>(n) * ld * es;

  cudaEvent_t ev0, ev1;
  SPX_CUDA(cudaEventCreate(&ev0));
  SPX_CUDA(cudaEventCreate(&ev1));
  SPX_CUDA(cudaEventRecord(ev0, st));
  if (o->precond == SPHYNX_PRECOND_POLY) poly_setup(g, o);
  if (o->precond == SPHYNX_PRECOND_AMG) amg_setup(g, o->seed, true);   // part of every partition, like the polynomial
  SPX_CUDA(cudaEventRecord(ev1, st));

  void *X[2] = {g->workspace("X0", blk, false), g->workspace("X1", blk, false)};
  void *LX[2] = {g->workspace("LX0", blk, false), g->workspace("LX1", blk, false)};
  void *P[2] = {g->workspace("P0", blk, true), g->workspace("P1", blk, true)};
  void *LP[2] = {g->workspace("LP0", blk, true), g->workspace("LP1", blk, true)};
  void *H = g->workspace("H", blk, true);
  void *LH = g->workspace("LH", blk, true);
  void *R = g->workspace("R", blk, true);
  const int ggrid = gram_grid(n), rgrid = residual_grid(n);
  double *gpart = static_cast<double *>(g->workspace("gram_part", gram_partials_size(3, ld, ggrid) * 8, false));
  const int M3 = 3 * ld;
  double *ga = static_cast<double *>(g->workspace("ga", M3 * M3 * 8, true));
  double *gb = static_cast<double *>(g->workspace("gb", M3 * M3 * 8, true));
  void *yt = g->workspace("yt", M3 * ld * es, true);
  double *npart = static_cast<double *>(g->workspace("npart", static_cast<size_t>(rgrid) * ld * 8, false));
  SolverState *state = static_cast<SolverState *>(g->workspace("state", sizeof(SolverState), true));
  const int *done = &state->done;
  const double *bd = gen ? g->deg.as<double>() : nullptr;
  const float *bdf = gen ? g->degf.as<float>() : nullptr;
  const bool jac = o->precond == SPHYNX_PRECOND_JACOBI && lap == SPHYNX_COMBINATORIAL;
  // the residual kernel writes H directly unless the polynomial or the multigrid cycle needs R
  const bool pre_r = o->precond == SPHYNX_PRECOND_POLY || o->precond == SPHYNX_PRECOND_AMG;
  void *res_out = pre_r ? R : H;
  // mixed precision with the polynomial: R is only the chain's input, whose
  // later vectors are stored in bfloat16 anyway, so the residual kernel
  // stores it in bfloat16 (its norms come from the float values) and the
  // first chain step gathers half the bytes
  const bool r_bf16 = o->precond == SPHYNX_PRECOND_POLY && o->precision == SPHYNX_MIXED_BF16 && g->poly_k >= 2;

  // initial block
  if (x0_host) {
    DevBuf tmp;
    tmp.alloc(static_cast<size_t>(n) * b * sizeof(double));
    SPX_CUDA(cudaMemcpyAsync(tmp.p, x0_host, static_cast<size_t>(n) * b * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_from_f64(st, dt, X[0], tmp.as<double>(), n, b, ld);
    SPX_CUDA(cudaStreamSynchronize(st));
  } else if (o->init == SPHYNX_INIT_PIECEWISE) {
    launch_piecewise_block(st, dt, X[0], n, b, ld, o->laplacian, g->deg.as<double>());
  } else {
    launch_random_block(st, dt, X[0], n, b, ld, o->seed);
  }
  // Rayleigh-Ritz on span(X~), then R = L X0 - B X0 Theta0
  plain_spmm(g, lap, dt, X[0], LX[0], ld, b, nullptr);
  GramArgs ga1{dt, 1, ld, n, {X[0], nullptr, nullptr}, {LX[0], nullptr, nullptr}, bd, bdf, gpart, ga, gb, done};
  const int pg1 = launch_gram(st, ga1, ggrid);
  launch_gram_reduce(st, gpart, 1, ld, pg1, ga, gb, done);
  launch_rayleigh_ritz(st, ga, gb, ld, ld, b, u_work, state, nullptr, yt, dt, nullptr, nullptr, nullptr,
                       o->precision != SPHYNX_FP64);
  UpdateArgs up1{dt, 1, ld, n, {X[0], nullptr, nullptr}, {nullptr, nullptr, nullptr}, yt, X[1], nullptr, nullptr, done};
  launch_update(st, up1);
  plain_spmm(g, lap, dt, X[1], LX[1], ld, b, done);
  ResidualArgs ra{dt, ld, n, X[1], LX[1], state->theta, bd, bdf, jac ? g->jinv.as<double>() : nullptr,
                  jac ? g->jinvf.as<float>() : nullptr, res_out, npart, done};
  ra.out_bf16 = r_bf16 ? 1 : 0;
  launch_residual(st, ra, rgrid);
  const int abs_test = o->conv == SPHYNX_CONV_ABS ? 1 : 0;
  launch_converge(st, state, npart, rgrid, b, ld, o->tol, floor_th, floor_res, 0, o->max_iter, 0, abs_test);
  g->ctr.launches += 8;

  int sync_every = o->sync_every;
  if (sync_every <= 0) sync_every = n >= (1 << 20) ? 1 : (n >= (1 << 17) ? 4 : 16);
  int cur = 1;
  int *hflag = static_cast<int *>(g->host_flag);
  for (int it = 0; it < o->max_iter; ++it) {
    const int nx = cur ^ 1;
    if (o->precond == SPHYNX_PRECOND_POLY) poly_apply(g, o->precision, R, H, ld, b, done, r_bf16);   // precondition
    if (o->precond == SPHYNX_PRECOND_AMG) amg_apply(g, dt, R, H, ld, done);
    plain_spmm(g, lap, dt, H, LH, ld, b, done);
    GramArgs g3{dt, 3, ld, n, {X[cur], H, P[cur]}, {LX[cur], LH, LP[cur]}, bd, bdf, gpart, ga, gb, done};
    const int pg3 = launch_gram(st, g3, ggrid);                                        // Rayleigh-Ritz
    launch_gram_reduce(st, gpart, 3, ld, pg3, ga, gb, done);
    launch_rayleigh_ritz(st, ga, gb, 3 * ld, ld, b, u_work, state, nullptr, yt, dt, nullptr, nullptr, nullptr,
                       o->precision != SPHYNX_FP64);
    UpdateArgs u3{dt, 3, ld, n, {X[cur], H, P[cur]}, {nullptr, LH, LP[cur]}, yt, X[nx], P[nx], LP[nx], done};
    launch_update(st, u3);                                                             // update, direction
    plain_spmm(g, lap, dt, X[nx], LX[nx], ld, b, done);                                 // residual
    ResidualArgs r3 = ra;
    r3.x = X[nx];
    r3.lx = LX[nx];
    launch_residual(st, r3, rgrid);
    launch_converge(st, state, npart, rgrid, b, ld, o->tol, floor_th, floor_res, 1, o->max_iter,
                    o->stall_window, abs_test);  // lock
    g->ctr.launches += 6;
    cur = nx;
    if ((it + 1) % sync_every == 0 || it + 1 == o->max_iter) {
      SPX_CUDA(cudaMemcpyAsync(hflag, done, sizeof(int), cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaStreamSynchronize(st));
      if (*hflag) break;
    }
  }
  SolverState hs;
  SPX_CUDA(cudaMemcpyAsync(&hs, state, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  EigenResult r;
  r.iterations = hs.iters;
  r.svqb = hs.svqb_steps;
  r.status = hs.done ? hs.status : (hs.nconv == b ? SPHYNX_OK : SPHYNX_ERR_NOCONV);
  if (!hs.done && o->max_iter == 0) r.status = hs.nconv == b ? SPHYNX_OK : SPHYNX_ERR_NOCONV;
  for (int j = 0; j < b; ++j) {
    r.theta[j] = hs.theta[j];
    r.res[j] = hs.resnorm[j];
  }
  r.x = X[(1 + hs.iters) & 1];
  r.dt = dt;
  r.ld = ld;
  SPX_CUDA(cudaEventElapsedTime(&r.ms_setup, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return r;
}

void begin_stats(sphynx_graph *g, bool timing) {
  g->ctr.launches = 0;
  g->ctr.spmm_launches = 0;
  g->ctr.spmm_bytes = 0;
  g->ctr.spmm_ms = 0;
  for (int i = 0; i < 3; ++i) {
    g->ctr.spmm_launches_dt[i] = 0;
    g->ctr.spmm_bytes_dt[i] = 0;
    g->ctr.spmm_ms_dt[i] = 0;
  }
  g->ctr.ev_used = 0;
  g->ctr.timing = timing;
}

void end_stats(sphynx_graph *g) {
  double ms = 0;
  for (size_t i = 0; i + 1 < g->ctr.ev_used; i += 2) {
    float t = 0;
    SPX_CUDA(cudaEventElapsedTime(&t, g->ctr.ev_pool[i], g->ctr.ev_pool[i + 1]));
    ms += t;
    g->ctr.spmm_ms_dt[g->ctr.ev_dt[i / 2]] += t;
  }
  g->ctr.spmm_ms = ms;
  g->ctr.timing = false;
}

void fill_stats(sphynx_graph *g, const EigenResult &r, int b, sphynx_stats *s) {
  s->status = r.status;
  s->iterations = r.iterations;
  s->nev = b;
  s->svqb_steps = r.svqb;
  for (int j = 0; j < SPHYNX_MAX_NEV; ++j) {
    s->eigenvalues[j] = j < b ? r.theta[j] : 0.0;
    s->resnorm[j] = j < b ? r.res[j] : 0.0;
  }
  s->ms_setup = r.ms_setup;
  s->ms_spmm = g->ctr.spmm_ms;
  s->spmm_launches = g->ctr.spmm_launches;
  s->spmm_bytes = g->ctr.spmm_bytes;
  for (int i = 0; i < 3; ++i) {
    s->ms_spmm_by_dt[i] = g->ctr.spmm_ms_dt[i];
    s->spmm_bytes_by_dt[i] = g->ctr.spmm_bytes_dt[i];
    s->spmm_launches_by_dt[i] = g->ctr.spmm_launches_dt[i];
  }
  s->kernel_launches = g->ctr.launches;
}

}  // namespace

void check_lobpcg_options(const sphynx_graph *g, const sphynx_options *o) { check_options(g, o); }

void canonical_rotation_block(sphynx_graph *g, void *x, int64_t rows, int ld, DT dt, const double *theta, int d,
                              double tol, uint64_t seed) {
  // runs of columns 1..d-1 whose neighbouring Ritz values differ by at most tol
  std::vector<std::pair<int, int>> runs;
  for (int j = 1; j < d;) {
    int k = j;
    while (k + 1 < d && std::fabs(theta[k + 1] - theta[k]) <=
                            tol * std::fmax(std::fabs(theta[k]), std::fabs(theta[k + 1])))
      ++k;
    if (k > j) runs.emplace_back(j, k);
    j = k + 1;
  }
  if (runs.empty() || rows < 1) return;
  cudaStream_t st = g->stream;
  const int grid = vec_grid(rows);
  double *part = static_cast<double *>(g->workspace("cr_part", static_cast<size_t>(vec_grid(g->n)) * SPHYNX_MAX_NEV * 8, false));
  double *mdev = static_cast<double *>(g->workspace("cr_m", SPHYNX_MAX_NEV * SPHYNX_MAX_NEV * 8, false));
  for (const auto &run : runs) {
    const int a = run.first, c = run.second - run.first + 1;
    for (int p = 0; p < c; ++p) {
      launch_cluster_dots(st, dt, x, rows, ld, d, a, c, p, seed, part, grid);
      launch_reduce_cols(st, part, grid, c, mdev + p * c);
      g->ctr.launches += 2;
    }
    std::vector<double> m(static_cast<size_t>(c) * c), s(static_cast<size_t>(c) * c), v, q(static_cast<size_t>(c) * c);
    SPX_CUDA(cudaMemcpyAsync(m.data(), mdev, m.size() * 8, cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    // S = M^T M = V diag(l) V^T, Q = M V diag(l^{-1/2}) V^T
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double acc = 0.0;
        for (int k = 0; k < c; ++k) acc += m[k * c + i] * m[k * c + j];
        s[i * c + j] = acc;
      }
    sym_eig_host(s, c, v);
    bool full_rank = true;
    for (int i = 0; i < c; ++i) full_rank = full_rank && s[i * c + i] > 0.0;
    if (!full_rank) continue;   // a rank-deficient alignment leaves the cluster as computed
    std::vector<double> w(static_cast<size_t>(c) * c);   // V diag(l^{-1/2}) V^T
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double acc = 0.0;
        for (int k = 0; k < c; ++k) acc += v[i * c + k] * v[j * c + k] / std::sqrt(s[k * c + k]);
        w[i * c + j] = acc;
      }
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) {
        double acc = 0.0;
        for (int k = 0; k < c; ++k) acc += m[i * c + k] * w[k * c + j];
        q[i * c + j] = acc;
      }
    SPX_CUDA(cudaMemcpyAsync(mdev, q.data(), q.size() * 8, cudaMemcpyHostToDevice, st));
    launch_rotate_cols(st, dt, x, rows, ld, a, c, mdev);
    SPX_CUDA(cudaStreamSynchronize(st));
    g->ctr.launches += 1;
  }
}

namespace {

}  // namespace

}  // namespace sphynx

using namespace sphynx;

extern "C" {

int sphynx_laplacian_apply(sphynx_handle g, int32_t laplacian, int32_t dtype, const void *x, int32_t ldx, void *y,
                           int32_t ldy, int32_t ncols) {
  return guarded([&]() -> int {
    if (!g || !x || !y) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (laplacian < 0 || laplacian > 2) fail(SPHYNX_ERR_INVALID_ARG, "laplacian %d", laplacian);
    if (dtype < 0 || dtype > 2) fail(SPHYNX_ERR_INVALID_ARG, "dtype %d", dtype);
    if (ncols < 1 || ncols > SPHYNX_MAX_NEV) fail(SPHYNX_ERR_INVALID_ARG, "ncols %d", ncols);
    const int bp = ncols == 1 && ldx == 1 && ldy == 1 ? 1 : round4(ncols);
    if (ldx < bp || ldy < bp) fail(SPHYNX_ERR_INVALID_ARG, "leading dimensions must be >= %d", bp);
    if (bp > 1) {
      const size_t es = dt_size(static_cast<DT>(dtype));
      const size_t os = dtype == SPHYNX_DT_F64 ? 8 : 4;
      const size_t align = dtype == SPHYNX_DT_BF16 ? 8 : 16;
      if ((reinterpret_cast<uintptr_t>(x) % align) || (ldx * es) % align || (reinterpret_cast<uintptr_t>(y) % 16) ||
          (ldy * os) % 16)
        fail(SPHYNX_ERR_INVALID_ARG, "blocks must be 16-byte aligned row by row");
    }
    if (laplacian != SPHYNX_COMBINATORIAL && g->isolated > 0) fail(SPHYNX_ERR_ISOLATED, "vertex without edges");
    // the SpMM reads X rows exactly bp apart: pack a wider X into scratch first
    if (ldx != bp) {
      const size_t es = dt_size(static_cast<DT>(dtype));
      void *packed = g->workspace("la_x", static_cast<size_t>(g->n) * bp * es, false);
      SPX_CUDA(cudaMemcpy2DAsync(packed, bp * es, x, static_cast<size_t>(ldx) * es, bp * es, g->n,
                                 cudaMemcpyDeviceToDevice, g->stream));
      x = packed;
      ldx = bp;
    }
    SpmmArgs a{};
    a.lap = op_of(laplacian);
    a.tin = static_cast<DT>(dtype);
    a.ld_x = ldx;
    a.ld_y = ldy;
    a.bp = bp;
    a.b_true = ncols;
    a.x = x;
    a.y = y;
    spmm(g, a);
    return SPHYNX_OK;
  });
}

int sphynx_poly_step(sphynx_handle g, int32_t laplacian, int32_t dtype_in, const void *t, int32_t dtype_out,
                     void *t_out, void *y, int32_t ld, int32_t ncols, double theta_cur, double theta_next,
                     int32_t yterms, int32_t first) {
  return guarded([&]() -> int {
    if (!g || !t || !t_out || !y) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (laplacian < 0 || laplacian > 2) fail(SPHYNX_ERR_INVALID_ARG, "laplacian %d", laplacian);
    if (dtype_in < 0 || dtype_in > 2 || dtype_out < 0 || dtype_out > 2)
      fail(SPHYNX_ERR_INVALID_ARG, "dtype %d -> %d", dtype_in, dtype_out);
    const bool ok_types = (dtype_in == SPHYNX_DT_F64 && dtype_out == SPHYNX_DT_F64) ||
                          (dtype_in == SPHYNX_DT_F32 && dtype_out != SPHYNX_DT_F64) ||
                          (dtype_in == SPHYNX_DT_BF16 && dtype_out == SPHYNX_DT_BF16);
    if (!ok_types) fail(SPHYNX_ERR_INVALID_ARG, "chain types %d -> %d", dtype_in, dtype_out);
    if (ncols < 1 || ncols > SPHYNX_MAX_NEV || ld != round4(ncols))
      fail(SPHYNX_ERR_INVALID_ARG, "ncols %d / ld %d (ld must be round4(ncols))", ncols, ld);
    if (!(theta_cur != 0.0) || !(theta_next != 0.0) || !std::isfinite(theta_cur) || !std::isfinite(theta_next))
      fail(SPHYNX_ERR_INVALID_ARG, "roots must be finite and nonzero");
    if (laplacian != SPHYNX_COMBINATORIAL && g->isolated > 0) fail(SPHYNX_ERR_ISOLATED, "vertex without edges");
    double *inv = static_cast<double *>(g->workspace("ps_inv", 4 * sizeof(double), false));
    float *invf = static_cast<float *>(g->workspace("ps_invf", 4 * sizeof(float), false));
    if (g->step_theta[0] != theta_cur || g->step_theta[1] != theta_next) {
      // a copy from pageable memory has left the host buffer when it returns
      const double hinv[2] = {1.0 / theta_cur, 1.0 / theta_next};
      const float hinvf[2] = {static_cast<float>(hinv[0]), static_cast<float>(hinv[1])};
      SPX_CUDA(cudaMemcpyAsync(inv, hinv, sizeof(hinv), cudaMemcpyHostToDevice, g->stream));
      SPX_CUDA(cudaMemcpyAsync(invf, hinvf, sizeof(hinvf), cudaMemcpyHostToDevice, g->stream));
      g->step_theta[0] = theta_cur;
      g->step_theta[1] = theta_next;
    }
    SpmmArgs a{};
    a.lap = op_of(laplacian);
    a.tin = static_cast<DT>(dtype_in);
    a.ld_x = ld;
    a.ld_y = ld;
    a.bp = ld;
    a.b_true = ncols;
    a.x = t;
    a.mode = 1;
    a.t_out = t_out;
    a.tout = static_cast<DT>(dtype_out);
    a.yacc = y;
    a.first = first;
    a.yterms = yterms;
    a.inv = inv;
    a.invf = invf;
    a.i_cur = 0;
    spmm(g, a);
    return SPHYNX_OK;
  });
}

int sphynx_precond_setup(sphynx_handle g, const sphynx_options *opt, double *roots_out) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    check_options(g, opt);
    if (opt->precond == SPHYNX_PRECOND_AMG) {
      amg_setup(g, opt->seed, true);
      return SPHYNX_OK;
    }
    if (opt->precond != SPHYNX_PRECOND_POLY) return SPHYNX_OK;
    poly_setup(g, opt);
    if (roots_out) {
      for (int i = 0; i < opt->poly_degree + SPHYNX_MAX_ADDED_ROOTS; ++i)
        roots_out[i] = i < g->poly_k ? g->poly_roots[i] : INFINITY;
    }
    return SPHYNX_OK;
  });
}

int sphynx_precond_apply(sphynx_handle g, const sphynx_options *opt, const void *r, void *h, int32_t ld,
                         int32_t ncols) {
  return guarded([&]() -> int {
    if (!g || !r || !h) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    check_options(g, opt);
    if (ncols < 1 || ncols > SPHYNX_MAX_NEV || ld < round4(ncols) || ld % 4)
      fail(SPHYNX_ERR_INVALID_ARG, "ncols %d / ld %d", ncols, ld);
    const DT dt = block_dt(opt->precision);
    const int lap = op_of(opt->laplacian);
    if (opt->precond == SPHYNX_PRECOND_POLY) {
      if (g->poly_k == 0 || g->poly_degree != opt->poly_degree || g->poly_laplacian != lap)
        fail(SPHYNX_ERR_INVALID_ARG, "polynomial not set up for these options");
      if (ld != round4(ncols)) fail(SPHYNX_ERR_INVALID_ARG, "polynomial apply needs ld = round4(ncols)");
      poly_apply(g, opt->precision, r, h, ld, ncols, nullptr);
      return SPHYNX_OK;
    }
    if (opt->precond == SPHYNX_PRECOND_AMG) {
      if (ld != round4(ncols)) fail(SPHYNX_ERR_INVALID_ARG, "multigrid apply needs ld = round4(ncols)");
      amg_setup(g, opt->seed, false);
      amg_apply(g, dt, r, h, ld, nullptr);
      return SPHYNX_OK;
    }
    // Jacobi (identity for L_N) or none: H = diag^{-1} R through the residual
    // kernel with X = 0 (R = LX - 0 = the input block)
    const size_t bytes = static_cast<size_t>(g->n) * ld * dt_size(dt);
    void *zero = g->workspace("pa_zero", bytes, true);
    double *theta = static_cast<double *>(g->workspace("pa_theta", 16 * 8, true));
    const int grid = residual_grid(g->n);
    double *np = static_cast<double *>(g->workspace("pa_np", static_cast<size_t>(grid) * ld * 8, false));
    const bool jac = opt->precond == SPHYNX_PRECOND_JACOBI && lap == SPHYNX_COMBINATORIAL;
    ResidualArgs ra{dt, ld, g->n, zero, r, theta, nullptr, nullptr, jac ? g->jinv.as<double>() : nullptr,
                    jac ? g->jinvf.as<float>() : nullptr, h, np, nullptr};
    launch_residual(g->stream, ra, grid);
    return SPHYNX_OK;
  });
}

int sphynx_amg_level(sphynx_handle g, int32_t level, sphynx_amg_level_info *info, int32_t *agg_out,
                     int64_t *row_ptr_out, int32_t *col_out, float *w_out) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    amg_level_info(g, level, info, agg_out, row_ptr_out, col_out, w_out);
    return SPHYNX_OK;
  });
}

int sphynx_eigensolve(sphynx_handle g, const sphynx_options *opt, int32_t nev, const double *x0, void *x_out,
                      int32_t ldx, double *theta_out, double *resnorm_out, sphynx_stats *stats) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    const auto t0 = std::chrono::steady_clock::now();
    begin_stats(g, stats != nullptr);
    EigenResult r = lobpcg(g, opt, nev, x0);
    if (x_out) {
      if (ldx < r.ld) fail(SPHYNX_ERR_INVALID_ARG, "ldx < %d", r.ld);
      SPX_CUDA(cudaMemcpy2DAsync(x_out, ldx * dt_size(r.dt), r.x, r.ld * dt_size(r.dt), r.ld * dt_size(r.dt), g->n,
                                 cudaMemcpyDeviceToDevice, g->stream));
    }
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    end_stats(g);
    if (theta_out) memcpy(theta_out, r.theta, nev * sizeof(double));
    if (resnorm_out) memcpy(resnorm_out, r.res, nev * sizeof(double));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      fill_stats(g, r, nev, stats);
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return r.status;
  });
}

int sphynx_partition(sphynx_handle g, int32_t K, const sphynx_options *opt, int32_t *part_out, double *cut_out,
                     double *imbalance_out, sphynx_stats *stats) {
  return guarded([&]() -> int {
    if (!g || !part_out) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
    if (!opt) fail(SPHYNX_ERR_INVALID_ARG, "options are NULL");
    const auto t0 = std::chrono::steady_clock::now();
    const bool dev_out = (opt->flags & SPHYNX_OUT_DEVICE) != 0;
    cudaStream_t st = g->stream;
    begin_stats(g, stats != nullptr);
    int32_t *dpart = dev_out ? part_out
                             : static_cast<int32_t *>(g->workspace("part", static_cast<size_t>(g->n) * 4, false));
    if (stats) memset(stats, 0, sizeof(*stats));
    if (K == 1) {   // one part: no eigensolve
      SPX_CUDA(cudaMemsetAsync(dpart, 0, static_cast<size_t>(g->n) * 4, st));
      if (!dev_out) SPX_CUDA(cudaMemcpyAsync(part_out, dpart, g->n * 4, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaStreamSynchronize(st));
      if (cut_out) *cut_out = 0.0;
      if (imbalance_out) *imbalance_out = 1.0;
      if (stats) stats->imbalance = 1.0;
      return SPHYNX_OK;
    }
    int d = 0;
    while ((1LL << (d + 1)) <= K) ++d;
    d += 1;                                    // Eq. 4: d = floor(log2 K) + 1
    cudaEvent_t e[4];
    for (auto &x : e) SPX_CUDA(cudaEventCreate(&x));
    SPX_CUDA(cudaEventRecord(e[0], st));
    EigenResult r = lobpcg(g, opt, d, nullptr);
    SPX_CUDA(cudaEventRecord(e[1], st));
    canonical_rotation_block(g, const_cast<void *>(r.x), g->n, r.ld, r.dt, r.theta, d, opt->tol, opt->seed);
    // Algorithm 2: coordinates from eigenvectors 2..d
    const size_t es = dt_size(r.dt);
    void *coords = g->workspace("coords", static_cast<size_t>(g->n) * (d - 1) * es + 16, false);
    double *sc = static_cast<double *>(g->workspace("signs", static_cast<size_t>(vec_grid(g->n)) * d * 3 * 8 + 16 * 8, false));
    launch_signs_coords(st, r.dt, r.x, g->n, r.ld, d, coords, sc);
    void *mjs = g->workspace("mj", mj_scratch_bytes(g->n, K, 1), false);
    run_mj_scratch(st, r.dt, coords, d - 1, d - 1, g->n, g->vw, K, dpart, &g->ctr, mjs, nullptr, 1);   // multi-jagged partition
    g->ctr.launches += 3;
    int refine_moves = 0;
    if (opt->refine_rounds > 0)   // greedy improvement of the cut (Sec. 7), within 1 % imbalance
      refine_partition(g, dpart, K, 0.01, opt->refine_rounds, kRefineMaxDegree, &refine_moves, nullptr);
    SPX_CUDA(cudaEventRecord(e[2], st));
    double cut = 0, cut2 = 0, imb = 0;
    eval_partition(g, dpart, K, &cut, &cut2, &imb);
    SPX_CUDA(cudaEventRecord(e[3], st));
    if (!dev_out) SPX_CUDA(cudaMemcpyAsync(part_out, dpart, static_cast<size_t>(g->n) * 4, cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    end_stats(g);
    if (cut_out) *cut_out = cut;
    if (imbalance_out) *imbalance_out = imb;
    if (stats) {
      fill_stats(g, r, d, stats);
      float a = 0, b = 0, c = 0;
      SPX_CUDA(cudaEventElapsedTime(&a, e[0], e[1]));
      SPX_CUDA(cudaEventElapsedTime(&b, e[1], e[2]));
      SPX_CUDA(cudaEventElapsedTime(&c, e[2], e[3]));
      stats->ms_lobpcg = a;
      stats->ms_mj = b;
      stats->ms_eval = c;
      stats->cut = cut;
      stats->cut_twice = cut2;
      stats->imbalance = imb;
      stats->refine_moves = refine_moves;
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    for (auto &x : e) cudaEventDestroy(x);
    return r.status;
  });
}

}  // extern "C"
