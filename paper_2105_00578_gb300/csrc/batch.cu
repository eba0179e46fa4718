// batch.cu -- many graphs partitioned in one call.
//
// The graphs arrive as one block-diagonal CSR: graph q owns rows
// [gptr[q], gptr[q + 1]) and its rows reference only columns inside that
// range.  Each graph gets its own LOBPCG (Algorithm 1) with its own Ritz
// values, convergence test and soft locking, its own embedding and its own
// multi-jagged partition into K parts (Algorithm 2), exactly as if it were
// partitioned alone.
//
// What acts row by row -- the Laplacian SpMM, the Jacobi scaling, the residual
// -- runs over the whole batch with the single-graph kernels' arithmetic.
// What reduces over rows -- the Gram matrices, the residual norms, the
// embedding signs -- runs over chunks of at most kBatchChunk rows that never
// straddle two graphs, followed by a per-graph reduction in a fixed order.
// Rayleigh-Ritz and the convergence test run one CTA per graph.  A converged
// graph drops out of every per-chunk kernel.
//
// The iteration body is captured once into a CUDA graph under a conditional
// WHILE node whose condition a device kernel sets (some graph not done and
// the cap not reached), so the whole batched eigensolve is one graph launch
// with no host round trip between iterations.
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace sphynx {

namespace {

// rows per chunk: large enough that a CTA's reduction and its partial
// outputs are paid for by many rows (with 1024-row chunks, the 2000-graph
// batch's 75,000 chunks made each reduction kernel launch-overhead-bound)
constexpr int kBatchChunk = 16384;
constexpr int kGramRows = 64;       // rows staged per step of the batched Gram kernel
constexpr int kGramThreads = 256;
// iterations without a 10 % residual gain (at the float rounding floor) after
// which a float-block graph moves on to FP64 blocks
constexpr int kPromoteWindow = 20;
// iterations without a 10 % residual gain, anywhere above the floor, after
// which a float graph is also handed to the FP64 phase: rounding in a float
// basis can leave the iterate drifting well above the floor
constexpr int kFloatStuckWindow = 100;

int round4(int b) { return (b + 3) & ~3; }

struct ChunkView {
  const int32_t *graph;   // [n_chunks] graph of each chunk
  const int64_t *begin;   // [n_chunks + 1] first row of each chunk (last entry: n)
  int n = 0;              // chunks
  const int32_t *act = nullptr;   // when set: the chunks of graphs still iterating, walked by a
  const int *nact = nullptr;      // fixed grid (their count in *nact)
};

// chunk walks of the iteration kernels: every chunk once (grid = chunks), or
// the active list with a fixed grid
__device__ __forceinline__ int cv_count(const ChunkView &cv) { return cv.act ? *cv.nact : cv.n; }
__device__ __forceinline__ int cv_chunk(const ChunkView &cv, int i) { return cv.act ? cv.act[i] : i; }

__device__ __forceinline__ bool chunk_done(const SolverState *st, int q) { return st[q].done != 0; }

// ---- initial block: the single-graph random block of every graph (local rows) ----
// (orig: the caller's vertex of each row when the batch is reordered, so that
// a vertex draws the same numbers in any row)
template <typename T>
__global__ void k_brandom(T *x, ChunkView cv, const int64_t *gptr, const int32_t *orig, int b, int ld,
                          uint64_t state) {
  const int c = blockIdx.x, q = cv.graph[c];
  const int64_t r0 = cv.begin[c], r1 = cv.begin[c + 1], base = gptr[q];
  for (int64_t e = r0 * ld + threadIdx.x; e < r1 * ld; e += blockDim.x) {
    const int64_t i = e / ld;
    const int j = static_cast<int>(e - i * ld);
    const int64_t v_id = orig ? static_cast<int64_t>(orig[i]) : i;
    double v = 0.0;
    if (j < b) v = splitmix_pm1(state, static_cast<uint64_t>((v_id - base) * b + j + 1));
    x[e] = static_cast<T>(v);
  }
}

// rows back to the caller's order: y[orig[r]] = x[r] (rows of ld values)
template <typename T>
__global__ void k_bto_caller(const int32_t *orig, const T *x, int64_t n, int ld, T *y) {
  const int64_t total = n * ld;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / ld;
    y[static_cast<int64_t>(orig[r]) * ld + (e - r * ld)] = x[e];
  }
}

// part ids in row order from the caller-order ones: p_row[r] = p_caller[orig[r]]
__global__ void k_bparts_to_rows(const int32_t *orig, const int32_t *p_caller, int64_t n, int32_t *p_row) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p_row[r] = p_caller[orig[r]];
}

// ---- Gram matrices per chunk -------------------------------------------------
// S = [X | H | P] (nb blocks of ld columns, M = nb * ld), LS likewise.  The
// chunk's partial upper triangles of S^T L S and S^T B S go to
// partials[chunk][2 * npairs] (A pairs first).  Rows are staged kGramRows at a
// time; a thread owns pairs tid, tid + 256, ... and sums a staged block in the
// block type, then adds it into FP64 accumulators.
template <typename T, int PPT>
__global__ void __launch_bounds__(kGramThreads)
k_bgram(ChunkView cv, const SolverState *states, int nb, int ld, const T *s0, const T *s1, const T *s2,
        const T *l0, const T *l1, const T *l2, const T *bdiag, double *partials) {
  extern __shared__ __align__(16) unsigned char smraw[];
  for (int ci = blockIdx.x; ci < cv_count(cv); ci += gridDim.x) {
  const int c = cv_chunk(cv, ci), q = cv.graph[c];
  if (chunk_done(states, q)) continue;
  const int M = nb * ld, npairs = M * (M + 1) / 2, ntot = 2 * npairs;
  T *ss = reinterpret_cast<T *>(smraw);                     // [kGramRows][M]
  T *sl = ss + kGramRows * M;                               // [kGramRows][M]
  T *sd = sl + kGramRows * M;                               // [kGramRows] B diagonal
  unsigned char *pi = reinterpret_cast<unsigned char *>(sd + kGramRows);   // pair -> (i, j)
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    int i = 0, rem = p;
    while (rem >= M - i) {
      rem -= M - i;
      ++i;
    }
    pi[2 * p] = static_cast<unsigned char>(i);
    pi[2 * p + 1] = static_cast<unsigned char>(i + rem);
  }
  double acc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) acc[k] = 0.0;
  const T *sb[3] = {s0, s1, s2}, *lb[3] = {l0, l1, l2};
  const int64_t r0 = cv.begin[c], r1 = cv.begin[c + 1];
  for (int64_t rs = r0; rs < r1; rs += kGramRows) {
    const int rows = static_cast<int>(r1 - rs < kGramRows ? r1 - rs : kGramRows);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * M; e += blockDim.x) {
      const int r = e / M, col = e % M, blk = col / ld, k = col % ld;
      const int64_t row = rs + r;
      ss[e] = sb[blk][row * ld + k];
      sl[e] = lb[blk][row * ld + k];
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) sd[r] = bdiag ? bdiag[rs + r] : T(1);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int p = threadIdx.x + k * kGramThreads;
      if (p >= ntot) break;
      const bool isb = p >= npairs;
      const int pp = isb ? p - npairs : p;
      const int i = pi[2 * pp], j = pi[2 * pp + 1];
      T s = T(0);
      if (isb) {
        for (int r = 0; r < rows; ++r) s += ss[r * M + i] * (sd[r] * ss[r * M + j]);
      } else {
        for (int r = 0; r < rows; ++r) s += ss[r * M + i] * sl[r * M + j];
      }
      acc[k] += static_cast<double>(s);
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * kGramThreads;
    if (p < ntot) partials[static_cast<int64_t>(c) * ntot + p] = acc[k];
  }
  __syncthreads();   // shared buffers are reused by the next chunk
  }
}

// per graph: G = sum over its chunks (in chunk order) of the partials, both
// triangles written from the upper one
__global__ void k_bgram_reduce(const int32_t *gchunk0, const SolverState *states, int M, const double *partials,
                               double *ga, double *gb) {
  const int q = blockIdx.x;
  if (states[q].done) return;
  const int npairs = M * (M + 1) / 2, ntot = 2 * npairs;
  const int c0 = gchunk0[q], c1 = gchunk0[q + 1];
  double *A = ga + static_cast<size_t>(q) * M * M, *B = gb + static_cast<size_t>(q) * M * M;
  for (int p = threadIdx.x; p < ntot; p += blockDim.x) {
    double s = 0.0;
    for (int c = c0; c < c1; ++c) s += partials[static_cast<int64_t>(c) * ntot + p];
    const bool isb = p >= npairs;
    int rem = isb ? p - npairs : p, i = 0;
    while (rem >= M - i) {
      rem -= M - i;
      ++i;
    }
    const int j = i + rem;
    double *G = isb ? B : A;
    G[i * M + j] = s;
    G[j * M + i] = s;
  }
}

// ---- update: X' = S Y, P' = [0 H P] Y, LP' = [0 LH LP] Y with each graph's Y ----
template <typename T, int LD, int NBLK>
__global__ void __launch_bounds__(256)
k_bupdate(ChunkView cv, const SolverState *states, const T *s0, const T *s1, const T *s2, const T *l1,
          const T *l2, const T *yall, T *xo, T *po, T *lpo) {
  constexpr int M = NBLK * LD;
  __shared__ T sy[M * LD];
  for (int ci = blockIdx.x; ci < cv_count(cv); ci += gridDim.x) {
  const int c = cv_chunk(cv, ci), q = cv.graph[c];
  if (chunk_done(states, q)) continue;
  const T *y = yall + static_cast<size_t>(q) * M * LD;   // Rayleigh-Ritz wrote M x LD per graph
  for (int i = threadIdx.x; i < M * LD; i += blockDim.x) sy[i] = y[i];
  __syncthreads();
  const T *srows[3] = {s0, s1, s2};
  const T *lrows[3] = {nullptr, l1, l2};
  for (int64_t row = cv.begin[c] + threadIdx.x; row < cv.begin[c + 1]; row += blockDim.x) {
    T x[LD], p[LD], lp[LD];
#pragma unroll
    for (int k = 0; k < LD; ++k) {
      x[k] = T(0);
      p[k] = T(0);
      lp[k] = T(0);
    }
#pragma unroll
    for (int blk = 0; blk < NBLK; ++blk) {
#pragma unroll 1
      for (int k = 0; k < LD; ++k) {
        const T v = srows[blk][row * LD + k];
        const T lv = blk > 0 ? lrows[blk][row * LD + k] : T(0);
        const T *yr = sy + (blk * LD + k) * LD;
#pragma unroll
        for (int cc = 0; cc < LD; ++cc) {
          x[cc] += v * yr[cc];
          if (blk > 0) {
            p[cc] += v * yr[cc];
            lp[cc] += lv * yr[cc];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < LD; ++k) xo[row * LD + k] = x[k];
    if constexpr (NBLK == 3) {
#pragma unroll
      for (int k = 0; k < LD; ++k) {
        po[row * LD + k] = p[k];
        lpo[row * LD + k] = lp[k];
      }
    }
  }
  __syncthreads();   // shared buffers are reused by the next chunk
  }
}

// ---- residual R = LX - B X Theta (times the Jacobi diagonal), per-chunk norms ----
template <typename T, int LD>
__global__ void __launch_bounds__(256)
k_bresidual(ChunkView cv, const SolverState *states, const T *x, const T *lx, const T *bdiag, const T *jinv,
            T *out, double *partials) {
  __shared__ double red[8][LD];
  for (int ci = blockIdx.x; ci < cv_count(cv); ci += gridDim.x) {
  const int c = cv_chunk(cv, ci), q = cv.graph[c];
  if (chunk_done(states, q)) continue;
  T th[LD];
#pragma unroll
  for (int k = 0; k < LD; ++k) th[k] = static_cast<T>(states[q].theta[k]);
  T acc[LD];
#pragma unroll
  for (int k = 0; k < LD; ++k) acc[k] = T(0);
  for (int64_t row = cv.begin[c] + threadIdx.x; row < cv.begin[c + 1]; row += blockDim.x) {
    const T bi = bdiag ? bdiag[row] : T(1);
    const T ib = bdiag ? T(1) / bi : T(1);
    const T sc = jinv ? jinv[row] : T(1);
#pragma unroll
    for (int k = 0; k < LD; ++k) {
      T r = lx[row * LD + k] - th[k] * (bi * x[row * LD + k]);
      acc[k] += r * r * ib;
      out[row * LD + k] = r * sc;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < LD; ++k) {
    double v = static_cast<double>(acc[k]);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < LD) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    partials[static_cast<int64_t>(c) * LD + threadIdx.x] = s;
  }
  __syncthreads();   // shared buffers are reused by the next chunk
  }
}

// ---- convergence per graph (the single-graph test), and the loop condition ----
// ctl[0]: graphs not done; ctl[1]: iterations of the batch loop
// floors per graph, as the single-graph test takes them from that graph alone:
// theta within 10 u rho (rho = 2 max weighted degree for L_C, else 2) and the
// residual within 10 u rho (max degree + 1)
__global__ void k_bconverge(const int32_t *gchunk0, SolverState *states, int count, const double *partials, int b,
                            int ld, double tol, double u_work, int rho_from_degree,
                            const unsigned long long *gmax, int count_iteration, int maxit, int stall_window,
                            int abs_test, int early_promote, int *ctl) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  SolverState *st = states + q;
  if (st->done) return;
  const int c0 = gchunk0[q], c1 = gchunk0[q + 1];
  const double rho = rho_from_degree ? 2.0 * __longlong_as_double(static_cast<long long>(gmax[2 * q + 1])) : 2.0;
  const double floor_th = 10.0 * u_work * rho;
  const double floor_res = floor_th * static_cast<double>(gmax[2 * q] + 1);
  int nconv = 0;
  bool at_floor = false;   // an unconverged column whose target lies below this precision's floor, reached
  for (int j = 0; j < b; ++j) {
    double tot = 0.0;
    for (int c = c0; c < c1; ++c) tot += partials[static_cast<int64_t>(c) * ld + j];
    const double res = sqrt(tot);
    st->resnorm[j] = res;
    const double th = fabs(st->theta[j]);
    const double target = abs_test ? tol : tol * th;
    const bool ok = (res <= target) || (th <= floor_th && res <= floor_res);
    st->conv[j] = ok ? 1 : 0;
    nconv += ok ? 1 : 0;
    // stored vectors carry a rounding of about u |x|, so their residual cannot
    // fall much below u rho: a target under that is out of reach here
    if (!ok && th > floor_th && target < u_work * rho && res <= floor_th) at_floor = true;
  }
  st->nconv = nconv;
  if (count_iteration) {
    st->iters += 1;
    st->pvalid = 1;
  }
  bool stalled = stall_check(st, b, stall_window, count_iteration, floor_th);
  if (early_promote && count_iteration && at_floor) stalled = true;
  if (early_promote && count_iteration && stall_window > 0 && nconv < b) {
    bool stuck = true;
    for (int j = 0; j < b; ++j)
      if (!st->conv[j]) stuck = stuck && st->since_best[j] >= kFloatStuckWindow;
    if (stuck) stalled = true;
  }
  if (nconv == b) {
    st->done = 1;
    st->status = SPHYNX_OK;
  } else if (st->iters >= maxit || stalled) {
    st->done = 1;
    st->status = SPHYNX_ERR_NOCONV;
    st->stalled = stalled ? 1 : 0;
  }
  if (st->done) atomicSub(&ctl[0], 1);
}

__global__ void k_bloop_condition(int *ctl, int maxit, cudaGraphConditionalHandle h) {
  ctl[1] += 1;
  cudaGraphSetConditional(h, (ctl[0] > 0 && ctl[1] < maxit) ? 1u : 0u);
}

// ---- embedding signs per graph and column: largest |x| positive (lowest row on ties) ----
template <typename T>
__global__ void k_bargmax(ChunkView cv, const T *x, int ld, int b, double *pval, int64_t *pidx) {
  __shared__ double sv[256], svv[256];
  __shared__ int64_t si[256];
  const int c = blockIdx.x;
  for (int col = 0; col < b; ++col) {
    double best = -1.0, bestv = 0.0;
    int64_t bidx = INT64_MAX;
    for (int64_t row = cv.begin[c] + threadIdx.x; row < cv.begin[c + 1]; row += blockDim.x) {
      const double v = static_cast<double>(x[row * ld + col]);
      const double m = fabs(v);
      if (m > best) {
        best = m;
        bestv = v;
        bidx = row;
      }
    }
    sv[threadIdx.x] = best;
    svv[threadIdx.x] = bestv;
    si[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double a = sv[threadIdx.x], o = sv[threadIdx.x + s];
        const int64_t ia = si[threadIdx.x], io = si[threadIdx.x + s];
        if (o > a || (o == a && io < ia)) {
          sv[threadIdx.x] = o;
          si[threadIdx.x] = io;
          svv[threadIdx.x] = svv[threadIdx.x + s];
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      pval[(static_cast<int64_t>(c) * b + col) * 2] = sv[0];
      pval[(static_cast<int64_t>(c) * b + col) * 2 + 1] = svv[0];
      pidx[static_cast<int64_t>(c) * b + col] = si[0];
    }
    __syncthreads();
  }
}

__global__ void k_bsigns(const int32_t *gchunk0, int count, int b, const double *pval, const int64_t *pidx,
                         double *sign) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count * b) return;
  const int q = t / b, col = t % b;
  double best = -1.0, bestv = 0.0;
  int64_t bidx = INT64_MAX;
  for (int c = gchunk0[q]; c < gchunk0[q + 1]; ++c) {
    const double m = pval[(static_cast<int64_t>(c) * b + col) * 2];
    const int64_t i = pidx[static_cast<int64_t>(c) * b + col];
    if (m > best || (m == best && i < bidx)) {
      best = m;
      bidx = i;
      bestv = pval[(static_cast<int64_t>(c) * b + col) * 2 + 1];
    }
  }
  sign[t] = bestv < 0.0 ? -1.0 : 1.0;
}

template <typename T>
__global__ void k_bcoords(ChunkView cv, const T *x, int ld, int b, const double *sign, T *coords) {
  const int c = blockIdx.x, q = cv.graph[c];
  const double *sg = sign + static_cast<size_t>(q) * b;
  const int dims = b - 1;
  for (int64_t e = cv.begin[c] * dims + threadIdx.x; e < cv.begin[c + 1] * dims; e += blockDim.x) {
    const int64_t i = e / dims;
    const int j = static_cast<int>(e - i * dims);
    const T v = x[i * ld + j + 1];
    coords[e] = sg[j + 1] < 0.0 ? -v : v;
  }
}

// ---- parts back to local ids, cut and part weights per graph ------------------
__global__ void __launch_bounds__(256)
k_beval(ChunkView cv, const int64_t *rp, const int32_t *col, const float *w, const int64_t *vw, int32_t *part,
        int K, int wscale, unsigned long long *cut2, long long *pw, unsigned *bad) {
  const int c = blockIdx.x, q = cv.graph[c];
  unsigned long long acc = 0;
  unsigned b = 0;
  const int32_t off = q * K;
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    const int32_t pi = part[i];
    if (pi < off || pi >= off + K) {
      b = 1;
      continue;
    }
    const long long wv = vw ? vw[i] : 1;
    atomicAdd(reinterpret_cast<unsigned long long *>(&pw[pi]), static_cast<unsigned long long>(wv));
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      if (part[col[e]] != pi) {
        if (w) acc += static_cast<unsigned long long>(llrint(ldexp(static_cast<double>(w[e]), wscale)));
        else acc += 1;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&cut2[q], acc);
  if (b) atomicOr(bad, 1u);
}

// local part ids: part -= q K (after the cut, which compares global ids)
__global__ void k_blocal(ChunkView cv, int32_t *part, int K) {
  const int c = blockIdx.x, q = cv.graph[c];
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) part[i] -= q * K;
}

// every column of a graph's rows lies inside the graph's own row range
__global__ void k_check_blocks(ChunkView cv, const int64_t *gptr, const int64_t *rp, const int32_t *col,
                               unsigned *bad) {
  const int c = blockIdx.x, q = cv.graph[c];
  const int64_t lo = gptr[q], hi = gptr[q + 1];
  unsigned b = 0;
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (col[e] < lo || col[e] >= hi) b = 1;
  if (b) atomicOr(bad, 1u);
}

// per-graph maxima over the rows of each chunk: entries per row (the most
// terms a row of L adds) and weighted degree (non-negative doubles order like
// their bit patterns)
__global__ void k_bgraph_max(ChunkView cv, const int64_t *rp, const double *deg, unsigned long long *gmax) {
  __shared__ unsigned long long red[2][32];
  const int c = blockIdx.x, q = cv.graph[c];
  unsigned long long md = 0, mw = 0;
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    const unsigned long long d = static_cast<unsigned long long>(rp[i + 1] - rp[i]);
    const unsigned long long w = static_cast<unsigned long long>(__double_as_longlong(deg[i]));
    md = d > md ? d : md;
    mw = w > mw ? w : mw;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, md, o), b = __shfl_xor_sync(0xffffffffu, mw, o);
    md = a > md ? a : md;
    mw = b > mw ? b : mw;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = md;
    red[1][w] = mw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) {
      md = red[0][k] > md ? red[0][k] : md;
      mw = red[1][k] > mw ? red[1][k] : mw;
    }
    atomicMax(&gmax[2 * q], md);
    atomicMax(&gmax[2 * q + 1], mw);
  }
}

ChunkView view_of(const sphynx_graph *g) {
  ChunkView v{g->batch.chunk_graph.as<int32_t>(), g->batch.chunk_begin.as<int64_t>()};
  v.n = static_cast<int>(g->batch.n_chunks);
  return v;
}

// the iteration kernels' view: the active-chunk list while one is kept
ChunkView iter_view_of(const sphynx_graph *g) {
  ChunkView v = view_of(g);
  if (g->batch.act_chunks.p) {
    v.act = g->batch.act_chunks.as<int32_t>();
    v.nact = g->batch.n_act.as<int>() + 1;
  }
  return v;
}

unsigned iter_grid(const sphynx_graph *g) {
  const int64_t nc = g->batch.n_chunks;
  return static_cast<unsigned>(g->batch.act_chunks.p && nc > 8 * kSmCount ? 8 * kSmCount : nc);
}

// ---- polynomial preconditioner of every graph (Sec. 5.2) ----------------------
// The single-graph setup restated per graph: k Lanczos steps on each graph's
// own L with two classical Gram-Schmidt passes against its basis (its
// normalised null vector in column 0), then its harmonic Ritz values in
// modified Leja order.  Dots reduce per chunk, then per graph over its
// chunks in chunk order.  The basis is column-major over all rows.

// the start vector: graph q's rows draw the single-graph stream at their local index
template <typename T>
__global__ void k_bz_start(ChunkView cv, const int64_t *gptr, const int32_t *orig, T *v, uint64_t state) {
  const int c = blockIdx.x, q = cv.graph[c];
  const int64_t base = gptr[q];
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    const int64_t v_id = orig ? static_cast<int64_t>(orig[i]) : i;
    v[i] = static_cast<T>(splitmix_pm1(state, static_cast<uint64_t>(v_id - base + 1)));
  }
}

__device__ __forceinline__ double null_entry(int lap, const double *deg, int64_t i) {
  return lap == SPHYNX_NORMALIZED ? sqrt(deg[i]) : 1.0;
}

// per chunk: z . v and z . z (z the null vector of L)
template <typename T>
__global__ void __launch_bounds__(256) k_bz_null_dots(ChunkView cv, const T *v, int lap, const double *deg,
                                                      double *partials) {
  __shared__ double r0[8], r1[8];
  const int c = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    const double z = null_entry(lap, deg, i);
    a0 += z * static_cast<double>(v[i]);
    a1 += z * z;
  }
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, off);
    a1 += __shfl_down_sync(0xffffffffu, a1, off);
  }
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = a0;
    r1[threadIdx.x >> 5] = a1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < 8; ++k) {
      s0 += r0[k];
      s1 += r1[k];
    }
    partials[2 * static_cast<int64_t>(c)] = s0;
    partials[2 * static_cast<int64_t>(c) + 1] = s1;
  }
}

// out[q][col] (row stride ostride) = sum over graph q's chunks, in chunk order,
// of partials[chunk][col], col < cols
__global__ void k_bz_reduce(const int32_t *gchunk0, int count, const double *partials, int cols, double *out,
                            int ostride) {
  const int q = blockIdx.x;
  for (int col = threadIdx.x; col < cols; col += blockDim.x) {
    double s = 0.0;
    for (int c = gchunk0[q]; c < gchunk0[q + 1]; ++c) s += partials[static_cast<int64_t>(c) * cols + col];
    out[static_cast<int64_t>(q) * ostride + col] = s;
  }
}

// v <- v - (z.v / z.z) z  (scal[q] = {z.v, z.z}, stride 2)
template <typename T>
__global__ void k_bz_null_axpy(ChunkView cv, T *v, int lap, const double *deg, const double *scal) {
  const int c = blockIdx.x, q = cv.graph[c];
  const double f = scal[2 * q] / scal[2 * q + 1];
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x)
    v[i] = static_cast<T>(static_cast<double>(v[i]) - f * null_entry(lap, deg, i));
}

// col = z / ||z||
template <typename T>
__global__ void k_bz_null_column(ChunkView cv, T *col, int lap, const double *deg, const double *scal) {
  const int c = blockIdx.x, q = cv.graph[c];
  const double f = 1.0 / sqrt(scal[2 * q + 1]);
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x)
    col[i] = static_cast<T>(null_entry(lap, deg, i) * f);
}

// per chunk: the dots of w with basis columns 0 .. j1 - 1, eight at a time
template <typename T>
__global__ void __launch_bounds__(256) k_bz_dots(ChunkView cv, const T *basis, int64_t ldv, int j1, const T *w,
                                                 double *partials) {
  __shared__ double red[8][8];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < j1; c0 += 8) {
    T acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = T(0);
    for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
      const T wv = w[i];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (c0 + k < j1) acc[k] = fma(basis[static_cast<int64_t>(c0 + k) * ldv + i], wv, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double d = static_cast<double>(acc[k]);
      for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
      if (lane == 0) red[k][warp] = d;
    }
    __syncthreads();
    if (threadIdx.x < 8 && c0 + static_cast<int>(threadIdx.x) < j1) {
      double s = 0.0;
      for (int k = 0; k < 8; ++k) s += red[threadIdx.x][k];
      partials[static_cast<int64_t>(c) * j1 + c0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// w <- w - V[:, :j1] h_q, and npart[chunk] = the chunk's part of ||w||^2
template <typename T>
__global__ void __launch_bounds__(256) k_bz_sub(ChunkView cv, const T *basis, int64_t ldv, int j1, T *w,
                                                const double *h, int hstride, double *npart) {
  __shared__ T sh[SPHYNX_MAX_POLY_DEGREE + 2];
  __shared__ double red[8];
  const int c = blockIdx.x, q = cv.graph[c];
  for (int k = threadIdx.x; k < j1; k += blockDim.x) sh[k] = static_cast<T>(h[static_cast<int64_t>(q) * hstride + k]);
  __syncthreads();
  T acc = T(0);
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    T v = w[i];
    for (int k = 0; k < j1; ++k) v -= basis[static_cast<int64_t>(k) * ldv + i] * sh[k];
    w[i] = v;
    acc += v * v;
  }
  double d = static_cast<double>(acc);
  for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    npart[c] = s;
  }
}

// v = w / sqrt(beta2_q) and V[:, col] = v (beta2 of graph q at beta2[q * bstride])
template <typename T>
__global__ void k_bz_next(ChunkView cv, const T *w, T *v, T *basis, int64_t ldv, int col, const double *beta2,
                          int bstride) {
  const int c = blockIdx.x, q = cv.graph[c];
  const T inv = static_cast<T>(1.0 / sqrt(beta2[static_cast<int64_t>(q) * bstride]));
  T *bc = basis + static_cast<int64_t>(col) * ldv;
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) {
    const T val = w[i] * inv;
    v[i] = val;
    bc[i] = val;
  }
}

// dst[q * dstride] = src[q * sstride] for every graph
__global__ void k_bz_take(int count, const double *src, int sstride, double *dst, int dstride) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) dst[static_cast<int64_t>(q) * dstride] = src[static_cast<int64_t>(q) * sstride];
}

__global__ void k_row_graph(ChunkView cv, int32_t *rg) {
  const int c = blockIdx.x, q = cv.graph[c];
  for (int64_t i = cv.begin[c] + threadIdx.x; i < cv.begin[c + 1]; i += blockDim.x) rg[i] = q;
}

template <typename T>
void batch_poly_setup_t(sphynx_graph *g, int k, int lap, uint64_t seed) {
  BatchInfo &B = g->batch;
  const int count = B.count;
  cudaStream_t st = g->stream;
  const int64_t n = g->n;
  const int64_t ldv = (n + 3) & ~static_cast<int64_t>(3);
  const unsigned cg = static_cast<unsigned>(B.n_chunks);
  const ChunkView cv = view_of(g);
  const int32_t *gc0 = B.graph_chunk0.as<int32_t>();
  const double *deg = g->deg.as<double>();
  T *V = static_cast<T *>(g->workspace("bz_V", static_cast<size_t>(ldv) * (k + 1) * sizeof(T), false));
  T *v = static_cast<T *>(g->workspace("bz_v", static_cast<size_t>(ldv) * sizeof(T), false));
  T *w = static_cast<T *>(g->workspace("bz_w", static_cast<size_t>(ldv) * sizeof(T), false));
  const int S = SPHYNX_MAX_POLY_DEGREE + SPHYNX_MAX_ADDED_ROOTS + 2;   // per-graph stride of the small arrays
  double *part = static_cast<double *>(g->workspace("bz_part", static_cast<size_t>(B.n_chunks) * S * 8, false));
  double *small = static_cast<double *>(g->workspace("bz_small", static_cast<size_t>(count) * S * 5 * 8, true));
  double *alpha = small, *beta2 = small + static_cast<size_t>(count) * S, *h = beta2 + static_cast<size_t>(count) * S;
  double *scal = h + static_cast<size_t>(count) * S, *roots = scal + static_cast<size_t>(count) * S;
  int *err = static_cast<int *>(g->workspace("bz_err", static_cast<size_t>(count) * 2 * sizeof(int), true));
  int *kout = err + count;
  // start vector, null column, projection, normalisation
  k_bz_start<T><<<cg, 256, 0, st>>>(cv, B.gptr.as<int64_t>(), B.orig.as<int32_t>(), v, mix64(seed + 3 * kGamma));
  SPX_LAUNCHED();
  k_bz_null_dots<T><<<cg, 256, 0, st>>>(cv, v, lap, deg, part);
  SPX_LAUNCHED();
  k_bz_reduce<<<count, 32, 0, st>>>(gc0, count, part, 2, scal, 2);
  SPX_LAUNCHED();
  k_bz_null_axpy<T><<<cg, 256, 0, st>>>(cv, v, lap, deg, scal);
  SPX_LAUNCHED();
  k_bz_null_column<T><<<cg, 256, 0, st>>>(cv, V, lap, deg, scal);
  SPX_LAUNCHED();
  k_bz_dots<T><<<cg, 256, 0, st>>>(cv, v, ldv, 1, v, part);
  SPX_LAUNCHED();
  k_bz_reduce<<<count, 32, 0, st>>>(gc0, count, part, 1, h, S);
  SPX_LAUNCHED();
  k_bz_next<T><<<cg, 256, 0, st>>>(cv, v, v, V, ldv, 1, h, S);
  SPX_LAUNCHED();
  g->ctr.launches += 9;
  for (int j = 0; j < k; ++j) {
    SpmmArgs a{};                                        // w = L v_j (every graph at once)
    a.lap = lap;
    a.tin = std::is_same<T, double>::value ? DT::F64 : DT::F32;
    a.ld_x = a.ld_y = a.bp = a.b_true = 1;
    a.x = v;
    a.y = w;
    spmm(g, a);
    for (int pass = 0; pass < 2; ++pass) {               // two Gram-Schmidt passes
      k_bz_dots<T><<<cg, 256, 0, st>>>(cv, V, ldv, j + 2, w, part);
      SPX_LAUNCHED();
      k_bz_reduce<<<count, 32, 0, st>>>(gc0, count, part, j + 2, h, S);
      SPX_LAUNCHED();
      if (pass == 0) {
        k_bz_take<<<(count + 127) / 128, 128, 0, st>>>(count, h + j + 1, S, alpha + j, S);
        SPX_LAUNCHED();
      }
      k_bz_sub<T><<<cg, 256, 0, st>>>(cv, V, ldv, j + 2, w, h, S, part);
      SPX_LAUNCHED();
    }
    k_bz_reduce<<<count, 32, 0, st>>>(gc0, count, part, 1, beta2 + j, S);   // beta_j^2 = ||w||^2
    SPX_LAUNCHED();
    if (j + 1 < k) {
      k_bz_next<T><<<cg, 256, 0, st>>>(cv, w, v, V, ldv, j + 2, beta2 + j, S);
      SPX_LAUNCHED();
    }
    g->ctr.launches += 9;
  }
  launch_harmonic_ritz_batch(st, alpha, beta2, k, count, S, roots, h, reinterpret_cast<float *>(scal), err, kout);
  g->ctr.launches += 3;
  // roots in application order -> per-graph 1/theta arrays of stride KS (double
  // and float), KS - 1 the largest root count; a graph with fewer roots has
  // 1/theta = 0 (an infinite root) on the steps beyond its own
  std::vector<double> hinv(static_cast<size_t>(count) * S);
  std::vector<int> herr(static_cast<size_t>(count) * 2);
  SPX_CUDA(cudaMemcpyAsync(hinv.data(), h, hinv.size() * 8, cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaMemcpyAsync(herr.data(), err, herr.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  int kmax = k;
  for (int q = 0; q < count; ++q) {
    if (herr[q]) fail(SPHYNX_ERR_BREAKDOWN, "polynomial setup of graph %d: Lanczos tridiagonal not positive definite "
                      "(%d)", q, herr[q]);
    kmax = std::max(kmax, herr[count + q]);
  }
  const int KS = kmax + 1;
  B.poly_inv.alloc(static_cast<size_t>(count) * KS * sizeof(double));
  B.poly_invf.alloc(static_cast<size_t>(count) * KS * sizeof(float));
  std::vector<double> inv(static_cast<size_t>(count) * KS);
  std::vector<float> invf(inv.size());
  for (int q = 0; q < count; ++q)
    for (int i = 0; i < KS; ++i) {
      inv[static_cast<size_t>(q) * KS + i] = hinv[static_cast<size_t>(q) * S + i];
      invf[static_cast<size_t>(q) * KS + i] = static_cast<float>(inv[static_cast<size_t>(q) * KS + i]);
    }
  SPX_CUDA(cudaMemcpyAsync(B.poly_inv.p, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, st));
  SPX_CUDA(cudaMemcpyAsync(B.poly_invf.p, invf.data(), invf.size() * 4, cudaMemcpyHostToDevice, st));
  SPX_CUDA(cudaStreamSynchronize(st));   // the host vectors above feed asynchronous copies
  B.poly_k = kmax;
  B.poly_lap = lap;
}

template <typename T>
void launch_bgram_t(cudaStream_t st, const sphynx_graph *g, const SolverState *states, int nb, int ld,
                    const void *const *s, const void *const *ls, const void *bdiag, double *partials) {
  const int M = nb * ld, ntot = M * (M + 1);
  const size_t sm = static_cast<size_t>(kGramRows) * (2 * M + 1) * sizeof(T) + static_cast<size_t>(ntot) + 16;
  const unsigned grid = iter_grid(g);
  const T *S[3] = {static_cast<const T *>(s[0]), static_cast<const T *>(s[1]), static_cast<const T *>(s[2])};
  const T *LS[3] = {static_cast<const T *>(ls[0]), static_cast<const T *>(ls[1]), static_cast<const T *>(ls[2])};
  const int ppt = (ntot + kGramThreads - 1) / kGramThreads;
#define SPX_BGRAM(P)                                                                                       \
  {                                                                                                        \
    SPX_CUDA(cudaFuncSetAttribute(k_bgram<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                  static_cast<int>(sm)));                                                  \
    k_bgram<T, P><<<grid, kGramThreads, sm, st>>>(iter_view_of(g), states, nb, ld, S[0], S[1], S[2], LS[0],    \
                                                  LS[1], LS[2], static_cast<const T *>(bdiag), partials); \
  }
  if (ppt <= 1) SPX_BGRAM(1)
  else if (ppt <= 2) SPX_BGRAM(2)
  else if (ppt <= 4) SPX_BGRAM(4)
  else if (ppt <= 10) SPX_BGRAM(10)
  else fail(SPHYNX_ERR_UNSUPPORTED, "batched Gram: block width %d too large", M);
#undef SPX_BGRAM
  SPX_LAUNCHED();
}

template <typename T, int LD>
void launch_bupdate_t(cudaStream_t st, const sphynx_graph *g, const SolverState *states, int nblk,
                      const void *const *s, const void *const *ls, const void *y, void *xo, void *po, void *lpo) {
  const unsigned grid = iter_grid(g);
  const T *S[3] = {static_cast<const T *>(s[0]), static_cast<const T *>(s[1]), static_cast<const T *>(s[2])};
  if (nblk == 1)
    k_bupdate<T, LD, 1><<<grid, 256, 0, st>>>(iter_view_of(g), states, S[0], nullptr, nullptr, nullptr, nullptr,
                                              static_cast<const T *>(y), static_cast<T *>(xo), nullptr, nullptr);
  else
    k_bupdate<T, LD, 3><<<grid, 256, 0, st>>>(iter_view_of(g), states, S[0], S[1], S[2],
                                              static_cast<const T *>(ls[1]), static_cast<const T *>(ls[2]),
                                              static_cast<const T *>(y), static_cast<T *>(xo), static_cast<T *>(po),
                                              static_cast<T *>(lpo));
  SPX_LAUNCHED();
}

template <typename T>
void launch_bupdate_ld(cudaStream_t st, const sphynx_graph *g, const SolverState *states, int ld, int nblk,
                       const void *const *s, const void *const *ls, const void *y, void *xo, void *po, void *lpo) {
  switch (ld) {
    case 4: launch_bupdate_t<T, 4>(st, g, states, nblk, s, ls, y, xo, po, lpo); break;
    case 8: launch_bupdate_t<T, 8>(st, g, states, nblk, s, ls, y, xo, po, lpo); break;
    case 12: launch_bupdate_t<T, 12>(st, g, states, nblk, s, ls, y, xo, po, lpo); break;
    case 16: launch_bupdate_t<T, 16>(st, g, states, nblk, s, ls, y, xo, po, lpo); break;
    default: fail(SPHYNX_ERR_UNSUPPORTED, "batched update: ld %d", ld);
  }
}

template <typename T>
void launch_bresidual_ld(cudaStream_t st, const sphynx_graph *g, const SolverState *states, int ld, const void *x,
                         const void *lx, const void *bdiag, const void *jinv, void *out, double *partials) {
  const unsigned grid = iter_grid(g);
  const T *X = static_cast<const T *>(x), *LX = static_cast<const T *>(lx);
  const T *B = static_cast<const T *>(bdiag), *J = static_cast<const T *>(jinv);
  T *O = static_cast<T *>(out);
  switch (ld) {
    case 4: k_bresidual<T, 4><<<grid, 256, 0, st>>>(iter_view_of(g), states, X, LX, B, J, O, partials); break;
    case 8: k_bresidual<T, 8><<<grid, 256, 0, st>>>(iter_view_of(g), states, X, LX, B, J, O, partials); break;
    case 12: k_bresidual<T, 12><<<grid, 256, 0, st>>>(iter_view_of(g), states, X, LX, B, J, O, partials); break;
    case 16: k_bresidual<T, 16><<<grid, 256, 0, st>>>(iter_view_of(g), states, X, LX, B, J, O, partials); break;
    default: fail(SPHYNX_ERR_UNSUPPORTED, "batched residual: ld %d", ld);
  }
  SPX_LAUNCHED();
}

}  // namespace

void batch_setup(sphynx_graph *g, const int64_t *h_gptr, int count) {
  BatchInfo &B = g->batch;
  B.count = count;
  B.h_gptr.assign(h_gptr, h_gptr + count + 1);
  std::vector<int32_t> cg;
  std::vector<int64_t> cb;
  std::vector<int32_t> c0(static_cast<size_t>(count) + 1);
  for (int q = 0; q < count; ++q) {
    c0[q] = static_cast<int32_t>(cg.size());
    for (int64_t r = h_gptr[q]; r < h_gptr[q + 1]; r += kBatchChunk) {
      cg.push_back(q);
      cb.push_back(r);
    }
  }
  c0[count] = static_cast<int32_t>(cg.size());
  cb.push_back(g->n);
  B.n_chunks = static_cast<int64_t>(cg.size());
  B.gptr.alloc((count + 1) * sizeof(int64_t));
  B.chunk_graph.alloc(cg.size() * sizeof(int32_t) + 4);
  B.chunk_begin.alloc(cb.size() * sizeof(int64_t));
  B.graph_chunk0.alloc(c0.size() * sizeof(int32_t));
  SPX_CUDA(cudaMemcpyAsync(B.gptr.p, h_gptr, (count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
  SPX_CUDA(cudaMemcpyAsync(B.chunk_graph.p, cg.data(), cg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  SPX_CUDA(cudaMemcpyAsync(B.chunk_begin.p, cb.data(), cb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
  SPX_CUDA(cudaMemcpyAsync(B.graph_chunk0.p, c0.data(), c0.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           g->stream));
  DevBuf bad;
  bad.alloc(sizeof(unsigned));
  SPX_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), g->stream));
  k_check_blocks<<<static_cast<unsigned>(B.n_chunks), 256, 0, g->stream>>>(view_of(g), B.gptr.as<int64_t>(),
                                                                          g->rowptr, g->col, bad.as<unsigned>());
  SPX_LAUNCHED();
  unsigned hb = 0;
  SPX_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(hb), cudaMemcpyDeviceToHost, g->stream));
  SPX_CUDA(cudaStreamSynchronize(g->stream));
  if (hb) fail(SPHYNX_ERR_INVALID_ARG, "a graph of the batch has an edge leaving its own vertex range");
  B.graph_max.alloc(static_cast<size_t>(count) * 2 * sizeof(unsigned long long));
  SPX_CUDA(cudaMemsetAsync(B.graph_max.p, 0, static_cast<size_t>(count) * 2 * sizeof(unsigned long long), g->stream));
  k_bgraph_max<<<static_cast<unsigned>(B.n_chunks), 256, 0, g->stream>>>(view_of(g), g->rowptr, g->deg.as<double>(),
                                                                       B.graph_max.as<unsigned long long>());
  SPX_LAUNCHED();
  // the graph of every row: the products skip finished graphs' rows and the
  // polynomial chain reads each row's own roots
  B.row_graph.alloc(static_cast<size_t>(g->n) * sizeof(int32_t));
  k_row_graph<<<static_cast<unsigned>(B.n_chunks), 256, 0, g->stream>>>(view_of(g), B.row_graph.as<int32_t>());
  SPX_LAUNCHED();
}

// the active lists: chunks whose graph still iterates, and 1024-row blocks
// holding a row of such a graph (a block spans at most a few graphs, each at
// least two rows; graphs lo .. hi of its first and last rows are checked).
// One block; the order of the lists does not matter, every consumer writes
// per-row or per-chunk outputs.
__global__ void __launch_bounds__(1024) k_build_lists(const SolverState *states, const int32_t *chunk_graph,
                                                      int n_chunks, const int32_t *row_graph, int64_t n,
                                                      int32_t *act_chunks, int32_t *act_blocks, int *n_act) {
  __shared__ int cb, cc;
  if (threadIdx.x == 0) {
    cb = 0;
    cc = 0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n_chunks; c += blockDim.x)
    if (!states[chunk_graph[c]].done) act_chunks[atomicAdd(&cc, 1)] = c;
  const int64_t nblk = (n + 1023) / 1024;
  for (int64_t bk = threadIdx.x; bk < nblk; bk += blockDim.x) {
    const int64_t r0 = bk * 1024, r1 = r0 + 1024 < n ? r0 + 1024 : n;
    const int glo = row_graph[r0], ghi = row_graph[r1 - 1];
    bool active = false;
    for (int q = glo; q <= ghi && !active; ++q) active = !states[q].done;
    if (active) act_blocks[atomicAdd(&cb, 1)] = static_cast<int32_t>(bk);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    n_act[0] = cb;
    n_act[1] = cc;
  }
}

// float blocks to double, every row
__global__ void k_widen(ChunkView cv, const float *x, int ld, double *y) {
  const int c = blockIdx.x;
  for (int64_t e = cv.begin[c] * ld + threadIdx.x; e < cv.begin[c + 1] * ld; e += blockDim.x)
    y[e] = static_cast<double>(x[e]);
}

// double blocks rounded to float, the rows of graphs still iterating
__global__ void k_narrow(ChunkView cv, const SolverState *states, const double *x, int ld, float *y) {
  const int c = blockIdx.x;
  if (states[cv.graph[c]].done) return;
  for (int64_t e = cv.begin[c] * ld + threadIdx.x; e < cv.begin[c + 1] * ld; e += blockDim.x)
    y[e] = static_cast<float>(x[e]);
}

// float blocks to double, the rows of graphs still iterating
__global__ void k_widen_active(ChunkView cv, const SolverState *states, const float *x, int ld, double *y) {
  const int c = blockIdx.x;
  if (states[cv.graph[c]].done) return;
  for (int64_t e = cv.begin[c] * ld + threadIdx.x; e < cv.begin[c + 1] * ld; e += blockDim.x)
    y[e] = static_cast<double>(x[e]);
}

// reopen the promoted graphs for the FP64 phase: not done, nothing converged,
// no search direction yet, stall bookkeeping cleared; their iteration counts
// go on; ctl[0] = graphs not done, ctl[1] = 0 (the loop's own count)
__global__ void k_bpromote(SolverState *states, int count, const char *promoted, int *ctl) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    ctl[1] = 0;
    int c = 0;
    for (int k = 0; k < count; ++k) c += promoted[k] ? 1 : 0;
    ctl[0] = c;
  }
  if (q >= count || !promoted[q]) return;
  SolverState *s = states + q;
  s->done = 0;
  s->status = SPHYNX_OK;
  s->nconv = 0;
  s->pvalid = 0;
  s->stalled = 0;
  for (int j = 0; j < SPHYNX_MAX_NEV; ++j) {
    s->conv[j] = 0;
    s->best_res[j] = 0.0;
    s->since_best[j] = 0;
  }
}

// The batched partition: every graph's LOBPCG in one captured graph launch,
// then the per-graph embedding, multi-jagged and metrics.
void batch_partition(sphynx_graph *g, int K, const sphynx_options *o, int32_t *dpart, double *cuts, double *imbs,
                     double *eigs, int32_t *iters, int32_t *status, sphynx_stats *stats) {
  BatchInfo &B = g->batch;
  const int count = B.count;
  if (o->precond == SPHYNX_PRECOND_AMG)
    fail(SPHYNX_ERR_UNSUPPORTED, "batched partitions take the Jacobi or polynomial preconditioner, or none");
  if (o->precond == SPHYNX_PRECOND_POLY && o->poly_degree < 2)
    fail(SPHYNX_ERR_UNSUPPORTED, "batched polynomial preconditioning needs degree >= 2");
  if (o->init != SPHYNX_INIT_RANDOM) fail(SPHYNX_ERR_UNSUPPORTED, "batched partitions start from the random block");
  for (int q = 0; q < count; ++q)
    if (B.h_gptr[q + 1] - B.h_gptr[q] < 2) fail(SPHYNX_ERR_INVALID_ARG, "graph %d of the batch has < 2 vertices", q);
  int d = 0;
  while ((1LL << (d + 1)) <= K) ++d;
  d += 1;                                       // Eq. 4
  if (K == 1) {
    SPX_CUDA(cudaMemsetAsync(dpart, 0, static_cast<size_t>(g->n) * 4, g->stream));
    for (int q = 0; q < count; ++q) {
      if (cuts) cuts[q] = 0.0;
      if (imbs) imbs[q] = 1.0;
      if (eigs) eigs[q] = 0.0;
      if (iters) iters[q] = 0;
      if (status) status[q] = SPHYNX_OK;
    }
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    return;
  }
  const int b = d;
  if (b > SPHYNX_MAX_NEV) fail(SPHYNX_ERR_UNSUPPORTED, "K too large for %d eigenvectors", SPHYNX_MAX_NEV);
  cudaStream_t st = g->stream;
  const int64_t n = g->n;
  const DT dt0 = o->precision == SPHYNX_FP64 ? DT::F64 : DT::F32;
  const int ld = round4(b), M3 = 3 * ld;
  const int lap = o->laplacian == SPHYNX_NORMALIZED ? SPHYNX_NORMALIZED : SPHYNX_COMBINATORIAL;
  const bool gen = o->laplacian == SPHYNX_GENERALIZED;
  const int rho_from_degree = lap == SPHYNX_COMBINATORIAL && !gen ? 1 : 0;        // noise floors, per graph
  const bool jac = o->precond == SPHYNX_PRECOND_JACOBI && lap == SPHYNX_COMBINATORIAL;
  const bool poly = o->precond == SPHYNX_PRECOND_POLY;
  const int64_t nch = B.n_chunks;
  if (poly) {   // every graph's polynomial (Sec. 5.2), set up anew as a single-graph partition does
    if (dt0 == DT::F64) batch_poly_setup_t<double>(g, o->poly_degree, lap, o->seed);
    else batch_poly_setup_t<float>(g, o->poly_degree, lap, o->seed);
  }
  const size_t ntot3 = static_cast<size_t>(M3) * (M3 + 1);
  double *gpart = static_cast<double *>(g->workspace("bgram_part", static_cast<size_t>(nch) * ntot3 * 8, false));
  double *ga = static_cast<double *>(g->workspace("bga", static_cast<size_t>(count) * M3 * M3 * 8, true));
  double *gb = static_cast<double *>(g->workspace("bgb", static_cast<size_t>(count) * M3 * M3 * 8, true));
  double *npart = static_cast<double *>(g->workspace("bnpart", static_cast<size_t>(nch) * ld * 8, false));
  SolverState *states =
      static_cast<SolverState *>(g->workspace("bstates", static_cast<size_t>(count) * sizeof(SolverState), true));
  int *ctl = static_cast<int *>(g->workspace("bctl", 4 * sizeof(int), false));
  // the m x m eigenproblems are FP64 solves; float blocks start them from a float Jacobi basis
  const int mixed0 = o->precision != SPHYNX_FP64;
  const int32_t *gc0 = B.graph_chunk0.as<int32_t>();
  const unsigned cgrid = static_cast<unsigned>(nch);
  const int hctl[4] = {count, 0, 0, 0};
  SPX_CUDA(cudaMemcpyAsync(ctl, hctl, sizeof(hctl), cudaMemcpyHostToDevice, st));
  const bool timing = g->ctr.timing;
  g->ctr.timing = false;   // per-launch events cannot live inside a captured loop
  const int64_t nblk = (n + 1023) / 1024;
  B.act_blocks.alloc(static_cast<size_t>(nblk) * sizeof(int32_t) + 4);
  B.act_chunks.alloc(static_cast<size_t>(nch) * sizeof(int32_t) + 4);
  B.n_act.alloc(4 * sizeof(int));
  auto build_lists = [&]() {
    k_build_lists<<<1, 1024, 0, st>>>(states, B.chunk_graph.as<int32_t>(), static_cast<int>(nch),
                                      B.row_graph.as<int32_t>(), n, B.act_chunks.as<int32_t>(),
                                      B.act_blocks.as<int32_t>(), B.n_act.as<int>());
    SPX_LAUNCHED();
  };

  // One precision phase of the batched eigensolve: blocks of type dt (chain
  // vectors of type ct), started from the random block or (warm) from the
  // blocks already in X[0], the graphs whose state is not done iterating.
  // Returns the blocks; a graph's Ritz vectors end in X[(1 + its phase
  // iterations) & 1].
  struct Blocks {
    void *X[2], *LX[2], *P[2], *LP[2], *H, *LH, *R, *chain[2], *yt;
  };
  // pt: the precision the preconditioner works in (its input and accumulator);
  // a preconditioner only shapes the search directions, so the FP64 phase
  // applies the polynomial in float and widens H (the eigenpairs' accuracy
  // rests on X, L X, the Gram matrices and the residual, all in dt)
  auto run_phase = [&](DT dt, DT ct, DT pt, const char *tag, bool warm, int window, int early) -> Blocks {
    const size_t es = dt_size(dt);
    const size_t blk = static_cast<size_t>(n) * ld * es;
    const double u_work = dt == DT::F64 ? 0x1.0p-53 : 0x1.0p-24;
    const int mixed = dt == DT::F64 ? 0 : mixed0;
    const std::string t(tag);
    Blocks k{};
    k.X[0] = g->workspace("X0" + t, blk, false);
    k.X[1] = g->workspace("X1" + t, blk, false);
    k.LX[0] = g->workspace("LX0" + t, blk, false);
    k.LX[1] = g->workspace("LX1" + t, blk, false);
    k.P[0] = g->workspace("P0" + t, blk, true);
    k.P[1] = g->workspace("P1" + t, blk, true);
    k.LP[0] = g->workspace("LP0" + t, blk, true);
    k.LP[1] = g->workspace("LP1" + t, blk, true);
    k.H = g->workspace("H" + t, blk, true);
    k.LH = g->workspace("LH" + t, blk, true);
    // the residual goes to H directly (Jacobi, none) or to R, from which the chain makes H
    k.R = poly ? g->workspace("bR" + t, blk, true) : k.H;
    void *R_lo = nullptr, *H_lo = nullptr;
    if (poly) {
      k.chain[0] = g->workspace("chain0" + t, static_cast<size_t>(n) * ld * dt_size(ct), false);
      k.chain[1] = g->workspace("chain1" + t, static_cast<size_t>(n) * ld * dt_size(ct), false);
      if (pt != dt) {
        R_lo = g->workspace("bR_lo" + t, static_cast<size_t>(n) * ld * dt_size(pt), false);
        H_lo = g->workspace("bH_lo" + t, static_cast<size_t>(n) * ld * dt_size(pt), false);
      }
    }
    k.yt = g->workspace("byt" + t, static_cast<size_t>(count) * M3 * ld * es, true);
    void **X = k.X, **LX = k.LX, **P = k.P, **LP = k.LP;
    void *H = k.H, *LH = k.LH, *R = k.R, *yt = k.yt;
    const void *bd = gen ? (dt == DT::F64 ? static_cast<const void *>(g->deg.p) : g->degf.p) : nullptr;
    const void *jv = jac ? (dt == DT::F64 ? static_cast<const void *>(g->jinv.p) : g->jinvf.p) : nullptr;

    auto gram = [&](int nb, const void *const *s, const void *const *ls) {
      if (dt == DT::F64) launch_bgram_t<double>(st, g, states, nb, ld, s, ls, bd, gpart);
      else launch_bgram_t<float>(st, g, states, nb, ld, s, ls, bd, gpart);
      k_bgram_reduce<<<count, 256, 0, st>>>(gc0, states, nb * ld, gpart, ga, gb);
      SPX_LAUNCHED();
    };
    auto update = [&](int nb, const void *const *s, const void *const *ls, void *xo, void *po, void *lpo) {
      if (dt == DT::F64) launch_bupdate_ld<double>(st, g, states, ld, nb, s, ls, yt, xo, po, lpo);
      else launch_bupdate_ld<float>(st, g, states, ld, nb, s, ls, yt, xo, po, lpo);
    };
    auto residual = [&](const void *x, const void *lx, void *out) {
      if (dt == DT::F64) launch_bresidual_ld<double>(st, g, states, ld, x, lx, bd, jv, out, npart);
      else launch_bresidual_ld<float>(st, g, states, ld, x, lx, bd, jv, out, npart);
    };
    auto converge = [&](int count_iteration) {
      k_bconverge<<<(count + 127) / 128, 128, 0, st>>>(gc0, states, count, npart, b, ld, o->tol, u_work,
                                                        rho_from_degree, B.graph_max.as<unsigned long long>(),
                                                        count_iteration, o->max_iter, window,
                                                        o->conv == SPHYNX_CONV_ABS ? 1 : 0, early, ctl);
      SPX_LAUNCHED();
      build_lists();   // graphs that finished drop out of the next iteration's launches
    };
    // H = p(L) R with each row's graph's roots: the single-graph product-form chain
    auto precondition = [&]() {
      if (!poly) return;
      const int kk = B.poly_k;
      const bool low = pt != dt;   // FP64 phase: the polynomial in float, H widened
      if (low) {
        k_narrow<<<cgrid, 256, 0, st>>>(view_of(g), states, static_cast<const double *>(R), ld,
                                        static_cast<float *>(R_lo));
        SPX_LAUNCHED();
      }
      for (int i = 0; i + 1 < kk; ++i) {
        SpmmArgs a{};
        a.lap = lap;
        a.tin = i == 0 ? pt : ct;
        a.ld_x = a.ld_y = a.bp = ld;
        a.b_true = b;
        a.x = i == 0 ? (low ? R_lo : R) : k.chain[(i - 1) & 1];
        a.mode = 1;
        a.t_out = k.chain[i & 1];
        a.tout = ct;
        a.yacc = low ? H_lo : H;
        a.first = i == 0 ? 1 : 0;
        a.yterms = (i % 2 == 0) ? 2 : (i + 2 == kk ? 1 : 0);
        a.inv = B.poly_inv.as<double>();
        a.invf = B.poly_invf.as<float>();
        a.i_cur = i;
        a.row_graph = B.row_graph.as<int32_t>();
        a.inv_stride = kk + 1;
        a.act_blocks = B.act_blocks.as<int32_t>();
        a.n_act = B.n_act.as<int>();
        spmm(g, a);
      }
      if (low) {
        k_widen_active<<<cgrid, 256, 0, st>>>(view_of(g), states, static_cast<const float *>(H_lo), ld,
                                              static_cast<double *>(H));
        SPX_LAUNCHED();
      }
    };
    auto spmm_block = [&](const void *x, void *y) {
      SpmmArgs a{};
      a.lap = lap;
      a.tin = dt;
      a.ld_x = ld;
      a.ld_y = ld;
      a.bp = ld;
      a.b_true = b;
      a.x = x;
      a.y = y;
      a.mode = 0;
      a.row_graph = B.row_graph.as<int32_t>();
      a.act_blocks = B.act_blocks.as<int32_t>();
      a.n_act = B.n_act.as<int>();
      spmm(g, a);
    };

    build_lists();   // the graphs this phase iterates
    // every graph's random block on its local rows (unless warm); then the
    // first Rayleigh-Ritz and residual
    if (!warm) {
      if (dt == DT::F64)
        k_brandom<double><<<cgrid, 256, 0, st>>>(static_cast<double *>(X[0]), view_of(g), B.gptr.as<int64_t>(),
                                                 B.orig.as<int32_t>(), b, ld, mix64(o->seed + kGamma));
      else
        k_brandom<float><<<cgrid, 256, 0, st>>>(static_cast<float *>(X[0]), view_of(g), B.gptr.as<int64_t>(),
                                                B.orig.as<int32_t>(), b, ld, mix64(o->seed + kGamma));
      SPX_LAUNCHED();
    }
    spmm_block(X[0], LX[0]);
    {
      // the first Rayleigh-Ritz: ld x ld problems per graph, back to back
      const void *s1[3] = {X[0], X[0], X[0]}, *l1[3] = {LX[0], LX[0], LX[0]};
      gram(1, s1, l1);
    }
    launch_rayleigh_ritz(st, ga, gb, ld, ld, b, u_work, states, nullptr, yt, dt, nullptr, nullptr, nullptr, mixed,
                         count);
    {
      const void *s1[3] = {X[0], nullptr, nullptr}, *l1[3] = {nullptr, nullptr, nullptr};
      update(1, s1, l1, X[1], nullptr, nullptr);
    }
    spmm_block(X[1], LX[1]);
    residual(X[1], LX[1], R);
    converge(0);
    SPX_CUDA(cudaStreamSynchronize(st));

    // the iteration body, captured once and repeated by a conditional WHILE node
    // (two bodies, one per ping-pong parity, so that a body is a fixed sequence)
    cudaGraph_t graph;
    SPX_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    SPX_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    SPX_CUDA(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    SPX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = g->stream;
    g->stream = cs;
    st = cs;
    try {
      SPX_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      for (int half = 0; half < 2; ++half) {   // X[1] -> X[0] -> X[1]: two iterations per body
        const int cur = half == 0 ? 1 : 0, nx = cur ^ 1;
        precondition();
        spmm_block(H, LH);
        const void *s3[3] = {X[cur], H, P[cur]}, *l3[3] = {LX[cur], LH, LP[cur]};
        gram(3, s3, l3);
        launch_rayleigh_ritz(st, ga, gb, M3, ld, b, u_work, states, nullptr, yt, dt, nullptr, nullptr, nullptr,
                             mixed, count);
        update(3, s3, l3, X[nx], P[nx], LP[nx]);
        spmm_block(X[nx], LX[nx]);
        residual(X[nx], LX[nx], R);
        converge(1);
      }
      k_bloop_condition<<<1, 1, 0, cs>>>(ctl, (o->max_iter + 1) / 2, cond);
      SPX_LAUNCHED();
      cudaGraph_t captured = nullptr;
      SPX_CUDA(cudaStreamEndCapture(cs, &captured));
    } catch (...) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cs, &junk);
      g->stream = saved;
      cudaStreamDestroy(cs);
      cudaGraphDestroy(graph);
      throw;
    }
    g->stream = saved;
    st = saved;
    cudaGraphExec_t exec;
    SPX_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    // the whole batched eigensolve of this phase: one launch
    SPX_CUDA(cudaGraphLaunch(exec, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return k;
  };

  // bring every graph's vectors of a phase into X[0] (rows of graphs whose
  // phase ended on X[1] copied over)
  auto gather_x0 = [&](const Blocks &k, DT dt, const std::vector<SolverState> &hs, const std::vector<int> &it0,
                       const std::vector<char> &take) {
    const size_t es = dt_size(dt);
    for (int q = 0; q < count; ++q) {
      if (!take[q] || ((1 + hs[q].iters - it0[q]) & 1) == 0) continue;
      const size_t off = static_cast<size_t>(B.h_gptr[q]) * ld * es;
      const size_t bytes = static_cast<size_t>(B.h_gptr[q + 1] - B.h_gptr[q]) * ld * es;
      SPX_CUDA(cudaMemcpyAsync(static_cast<char *>(k.X[0]) + off, static_cast<const char *>(k.X[1]) + off, bytes,
                               cudaMemcpyDeviceToDevice, st));
    }
  };
  auto read_states = [&]() {
    std::vector<SolverState> hs(count);
    SPX_CUDA(cudaMemcpyAsync(hs.data(), states, count * sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    return hs;
  };

  // Phase 1 in the requested precision.  Float blocks cannot resolve a
  // residual below about u ||L|| (the rounding of the stored vectors), and
  // tol |theta_2| lies below that on large graphs with small eigenvalues:
  // such a graph stops once a column whose target is below u rho has reached
  // the floor region (residual <= 10 u rho), or once it stalls (the stall
  // window), and finishes in FP64 blocks, warm-started from its float iterate.
  const bool promote = dt0 != DT::F64;
  const int window1 = promote ? (o->stall_window > 0 ? o->stall_window : kPromoteWindow) : o->stall_window;
  const DT ct0 = o->precision == SPHYNX_FP64 ? DT::F64 : (o->precision == SPHYNX_MIXED_BF16 ? DT::BF16 : DT::F32);
  auto tp = std::chrono::steady_clock::now();
  Blocks k1 = run_phase(dt0, ct0, dt0, "", false, window1, promote ? 1 : 0);
  double ms_phase[2] = {std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp).count(), 0.0};
  int loop_bodies[2] = {0, 0};   // each captured body runs two iterations
  SPX_CUDA(cudaMemcpyAsync(&loop_bodies[0], ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<SolverState> hs = read_states();
  std::vector<int> zero_it(count, 0);
  std::vector<char> all(count, 1);
  gather_x0(k1, dt0, hs, zero_it, all);
  DT dt = dt0;
  void *EX = k1.X[0];   // the final Ritz vectors of every graph (n x ld, type dt)
  std::vector<char> promoted(count, 0);
  int n_promoted = 0;
  if (promote) {
    for (int q = 0; q < count; ++q)
      if (hs[q].status != SPHYNX_OK && hs[q].iters < o->max_iter) {
        promoted[q] = 1;
        ++n_promoted;
      }
  }
  if (n_promoted > 0) {
    std::vector<int> it1(count);
    for (int q = 0; q < count; ++q) it1[q] = hs[q].iters;
    // every graph's float vectors widened to double; the promoted graphs resume from theirs
    const size_t blk64 = static_cast<size_t>(n) * ld * 8;
    double *X64 = static_cast<double *>(g->workspace("X0_64", blk64, false));
    k_widen<<<cgrid, 256, 0, st>>>(view_of(g), static_cast<const float *>(EX), ld, X64);
    SPX_LAUNCHED();
    DevBuf dprom;
    dprom.alloc(static_cast<size_t>(count));
    SPX_CUDA(cudaMemcpyAsync(dprom.p, promoted.data(), static_cast<size_t>(count), cudaMemcpyHostToDevice, st));
    k_bpromote<<<(count + 127) / 128, 128, 0, st>>>(states, count, dprom.as<char>(), ctl);
    SPX_LAUNCHED();
    SPX_CUDA(cudaStreamSynchronize(st));   // `promoted` feeds an asynchronous copy
    tp = std::chrono::steady_clock::now();
    Blocks k2 = run_phase(DT::F64, ct0, DT::F32, "_64", true, o->stall_window, 0);
    ms_phase[1] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp).count();
    SPX_CUDA(cudaMemcpyAsync(&loop_bodies[1], ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    hs = read_states();
    gather_x0(k2, DT::F64, hs, it1, promoted);
    dt = DT::F64;
    EX = k2.X[0];
  }
  const size_t es = dt_size(dt);
  g->ctr.timing = timing;
  B.act_blocks.release();   // the lists serve the iteration loops only
  B.act_chunks.release();
  B.n_act.release();
  // a reordered batch: the Ritz vectors back to the caller's order, where the
  // embedding and multi-jagged run exactly as on the caller's numbering (their
  // ties go to the lowest vertex id)
  const int32_t *orig = B.orig.as<int32_t>();
  if (orig) {
    void *EXc = g->workspace("EX_caller", static_cast<size_t>(n) * ld * es, false);
    const unsigned gr = static_cast<unsigned>(std::min<int64_t>((n * ld + 255) / 256, 16 * kSmCount));
    if (dt == DT::F64)
      k_bto_caller<double><<<gr, 256, 0, st>>>(orig, static_cast<const double *>(EX), n, ld, static_cast<double *>(EXc));
    else
      k_bto_caller<float><<<gr, 256, 0, st>>>(orig, static_cast<const float *>(EX), n, ld, static_cast<float *>(EXc));
    SPX_LAUNCHED();
    EX = EXc;
  }

  for (int q = 0; q < count; ++q) {
    const int64_t r0 = B.h_gptr[q], rows = B.h_gptr[q + 1] - r0;
    canonical_rotation_block(g, static_cast<char *>(EX) + static_cast<size_t>(r0) * ld * es, rows, ld, dt,
                             hs[q].theta, d, o->tol, o->seed);
  }
  // embedding (Algorithm 2), signs per graph
  double *pval = static_cast<double *>(g->workspace("bsg_val", static_cast<size_t>(nch) * b * 2 * 8, false));
  int64_t *pidx = static_cast<int64_t *>(g->workspace("bsg_idx", static_cast<size_t>(nch) * b * 8, false));
  double *sign = static_cast<double *>(g->workspace("bsg", static_cast<size_t>(count) * b * 8, false));
  void *coords = g->workspace("coords", static_cast<size_t>(n) * (d - 1) * es + 16, false);
  if (dt == DT::F64) k_bargmax<double><<<cgrid, 256, 0, st>>>(view_of(g), static_cast<const double *>(EX), ld, b, pval, pidx);
  else k_bargmax<float><<<cgrid, 256, 0, st>>>(view_of(g), static_cast<const float *>(EX), ld, b, pval, pidx);
  SPX_LAUNCHED();
  k_bsigns<<<(count * b + 255) / 256, 256, 0, st>>>(gc0, count, b, pval, pidx, sign);
  SPX_LAUNCHED();
  if (dt == DT::F64)
    k_bcoords<double><<<cgrid, 256, 0, st>>>(view_of(g), static_cast<const double *>(EX), ld, b, sign,
                                             static_cast<double *>(coords));
  else
    k_bcoords<float><<<cgrid, 256, 0, st>>>(view_of(g), static_cast<const float *>(EX), ld, b, sign,
                                            static_cast<float *>(coords));
  SPX_LAUNCHED();
  // multi-jagged over all graphs at once: graph q owns parts [q K, (q + 1) K)
  const int ktot = count * K;
  void *mjs = g->workspace("mj", mj_scratch_bytes(n, ktot, count), false);
  const int64_t *vw_caller = orig && B.vw_orig.p ? B.vw_orig.as<int64_t>() : g->vw;
  run_mj_scratch(st, dt, coords, d - 1, d - 1, n, vw_caller, ktot, dpart, &g->ctr, mjs, B.h_gptr.data(), count);
  // metrics per graph
  if (g->weighted && !g->wexact)
    fail(SPHYNX_ERR_UNSUPPORTED, "edge weights span too many binary orders for an exact cut");
  const size_t need = 64 + static_cast<size_t>(count) * 8 + static_cast<size_t>(ktot) * 8;
  char *ws = static_cast<char *>(g->workspace("beval", need, false));
  SPX_CUDA(cudaMemsetAsync(ws, 0, need, st));
  unsigned *dbad = reinterpret_cast<unsigned *>(ws);
  unsigned long long *dcut = reinterpret_cast<unsigned long long *>(ws + 64);
  long long *dpw = reinterpret_cast<long long *>(ws + 64 + static_cast<size_t>(count) * 8);
  int32_t *prow = dpart;   // the part of every row, in the handle's row order
  if (orig) {
    prow = static_cast<int32_t *>(g->workspace("bparts_rows", static_cast<size_t>(n) * sizeof(int32_t), false));
    k_bparts_to_rows<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 16 * kSmCount)), 256, 0, st>>>(
        orig, dpart, n, prow);
    SPX_LAUNCHED();
  }
  k_beval<<<cgrid, 256, 0, st>>>(view_of(g), g->rowptr, g->col, g->w, g->vw, prow, K, g->wscale, dcut, dpw, dbad);
  SPX_LAUNCHED();
  k_blocal<<<cgrid, 256, 0, st>>>(view_of(g), dpart, K);
  SPX_LAUNCHED();
  std::vector<char> host(need);
  SPX_CUDA(cudaMemcpyAsync(host.data(), ws, need, cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  unsigned hbad;
  memcpy(&hbad, host.data(), sizeof(hbad));
  if (hbad) fail(SPHYNX_ERR_INVALID_ARG, "batched multi-jagged produced a part outside its graph");
  const unsigned long long *hcut = reinterpret_cast<const unsigned long long *>(host.data() + 64);
  const long long *hpw = reinterpret_cast<const long long *>(host.data() + 64 + static_cast<size_t>(count) * 8);
  int nconv_graphs = 0;
  for (int q = 0; q < count; ++q) {
    long long mx = 0, tot = 0;
    for (int k = 0; k < K; ++k) {
      const long long v = hpw[static_cast<size_t>(q) * K + k];
      mx = v > mx ? v : mx;
      tot += v;
    }
    if (cuts) cuts[q] = ldexp(static_cast<double>(hcut[q]), g->weighted ? -(g->wscale + 1) : -1);
    if (imbs) imbs[q] = (static_cast<double>(mx) * static_cast<double>(K)) / static_cast<double>(tot);
    if (iters) iters[q] = hs[q].iters;
    if (eigs)
      for (int j = 0; j < d; ++j) eigs[static_cast<size_t>(q) * d + j] = hs[q].theta[j];
    const int sq = hs[q].done ? hs[q].status : SPHYNX_ERR_NOCONV;
    if (status) status[q] = sq;
    nconv_graphs += sq == SPHYNX_OK ? 1 : 0;
  }
  if (stats) {
    int maxit = 0;
    for (int q = 0; q < count; ++q) maxit = std::max(maxit, hs[q].iters);
    stats->status = nconv_graphs == count ? SPHYNX_OK : SPHYNX_ERR_NOCONV;
    stats->fp64_finished = n_promoted;
    stats->ms_phase[0] = ms_phase[0];
    stats->ms_phase[1] = ms_phase[1];
    stats->loop_iters[0] = 2 * loop_bodies[0];
    stats->loop_iters[1] = 2 * loop_bodies[1];
    stats->iterations = maxit;
    stats->nev = b;
  }
}

}  // namespace sphynx

namespace sphynx {
void batch_parts_to_rows(sphynx_graph *g, const int32_t *p_caller, int32_t *p_rows) {
  const int64_t n = g->n;
  k_bparts_to_rows<<<static_cast<unsigned>(std::min<int64_t>((n + 255) / 256, 16 * kSmCount)), 256, 0, g->stream>>>(
      g->batch.orig.as<int32_t>(), p_caller, n, p_rows);
  SPX_LAUNCHED();
}
}  // namespace sphynx

namespace sphynx {
namespace {

// Run f(q) for q in [0, count) on the host's cores, graphs handed out in order.
template <class F>
void for_each_graph(int count, F f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = static_cast<int>(std::min<unsigned>(hw, static_cast<unsigned>(count)));
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int q = next++; q < count; q = next++) f(q);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
}

// Reverse Cuthill-McKee order of the vertices [g0, g1) of one graph, into
// order[g0 .. g1): a breadth-first order from a pseudo-peripheral vertex
// (the minimum-degree vertex of the last level of a search, twice, from the
// component's lowest vertex), neighbours taken by increasing degree (lowest
// id on ties), every component in turn, then reversed.
// Edges that leave the range are ignored here (create rejects them later).
void rcm_graph(const int64_t *rp, const int32_t *col, int64_t g0, int64_t g1, std::vector<char> &seen,
               int32_t *order) {
  const int64_t nl = g1 - g0;
  auto deg = [&](int64_t v) { return rp[v + 1] - rp[v]; };
  std::vector<int32_t> queue;
  queue.reserve(static_cast<size_t>(nl));
  std::vector<std::pair<int64_t, int32_t>> nb;
  // breadth-first levels from s over unvisited vertices, marking with `mark`; returns the last level's start
  auto bfs_last = [&](int32_t s, char mark) {
    queue.clear();
    queue.push_back(s);
    seen[s] = mark;
    size_t head = 0, level = 0;
    while (head < queue.size()) {
      level = head;
      const size_t end = queue.size();
      for (; head < end; ++head) {
        const int32_t v = queue[head];
        for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
          const int32_t u = col[k];
          if (u < g0 || u >= g1 || seen[u] == mark || seen[u] == 2) continue;
          seen[u] = mark;
          queue.push_back(u);
        }
      }
    }
    return level;
  };
  int64_t placed = 0;
  for (int64_t cursor = g0; cursor < g1; ++cursor) {
    if (seen[cursor] == 2) continue;
    int32_t s = static_cast<int32_t>(cursor);   // a vertex of the next component
    for (int pass = 0; pass < 2; ++pass) {
      const char mark = static_cast<char>(3 + pass);
      const size_t lv = bfs_last(s, mark);
      int32_t best = queue[lv];
      for (size_t i = lv; i < queue.size(); ++i)
        if (deg(queue[i]) < deg(best) || (deg(queue[i]) == deg(best) && queue[i] < best)) best = queue[i];
      for (int32_t v : queue) seen[v] = 0;
      s = best;
    }
    // Cuthill-McKee from s
    size_t head = static_cast<size_t>(placed);
    order[g0 + placed++] = s;
    seen[s] = 2;
    while (head < static_cast<size_t>(placed)) {
      const int32_t v = order[g0 + head++];
      nb.clear();
      for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
        const int32_t u = col[k];
        if (u < g0 || u >= g1 || seen[u] == 2) continue;
        seen[u] = 2;
        nb.emplace_back(deg(u), u);
      }
      std::sort(nb.begin(), nb.end());
      for (const auto &e : nb) order[g0 + placed++] = e.second;
    }
  }
  std::reverse(order + g0, order + g1);
}

// The batch in reverse Cuthill-McKee order: rows permuted within each graph
// (order[r] = the caller's vertex at row r), columns renumbered and sorted in
// each row, weights carried along.
struct PermutedCsr {
  std::vector<int32_t> order;
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<float> w;
  std::vector<int64_t> vw;
};

PermutedCsr permute_batch(const int64_t *rp, const int32_t *col, const float *w, const int64_t *vw,
                          const int64_t *gptr, int count, int64_t n) {
  PermutedCsr P;
  P.order.resize(static_cast<size_t>(n));
  std::vector<char> seen(static_cast<size_t>(n), 0);
  for_each_graph(count, [&](int q) { rcm_graph(rp, col, gptr[q], gptr[q + 1], seen, P.order.data()); });
  std::vector<int32_t> pos(static_cast<size_t>(n));
  for (int64_t r = 0; r < n; ++r) pos[P.order[r]] = static_cast<int32_t>(r);
  P.rp.resize(static_cast<size_t>(n) + 1);
  P.rp[0] = 0;
  for (int64_t r = 0; r < n; ++r) P.rp[r + 1] = P.rp[r] + (rp[P.order[r] + 1] - rp[P.order[r]]);
  const int64_t nnz = P.rp[n];
  P.col.resize(static_cast<size_t>(nnz));
  if (w) P.w.resize(static_cast<size_t>(nnz));
  if (vw) {
    P.vw.resize(static_cast<size_t>(n));
    for (int64_t r = 0; r < n; ++r) P.vw[r] = vw[P.order[r]];
  }
  for_each_graph(count, [&](int q) {
    std::vector<std::pair<int32_t, float>> row;
    for (int64_t r = gptr[q]; r < gptr[q + 1]; ++r) {
      const int32_t v = P.order[r];
      row.clear();
      for (int64_t k = rp[v]; k < rp[v + 1]; ++k) row.emplace_back(pos[col[k]], w ? w[k] : 0.f);
      std::sort(row.begin(), row.end(), [](const std::pair<int32_t, float> &a, const std::pair<int32_t, float> &b) {
        return a.first < b.first;
      });
      int64_t o = P.rp[r];
      for (const auto &e : row) {
        P.col[o] = e.first;
        if (w) P.w[o] = e.second;
        ++o;
      }
    }
  });
  return P;
}

}  // namespace
}  // namespace sphynx

using namespace sphynx;

extern "C" int sphynx_create_batch(const int64_t *row_ptr, const int32_t *col, const float *edge_w,
                                   const int64_t *vtx_w, const int64_t *graph_ptr, int32_t count, int64_t n,
                                   int64_t nnz, uint32_t flags, void *stream, sphynx_handle *out) {
  return guarded([&]() -> int {
    if (!out) fail(SPHYNX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!graph_ptr || count < 1) fail(SPHYNX_ERR_INVALID_ARG, "graph offsets missing or count < 1");
    if (graph_ptr[0] != 0 || graph_ptr[count] != n) fail(SPHYNX_ERR_INVALID_ARG, "graph offsets must span [0, n)");
    for (int q = 0; q < count; ++q)
      if (graph_ptr[q + 1] <= graph_ptr[q]) fail(SPHYNX_ERR_INVALID_ARG, "graph %d of the batch is empty", q);
    sphynx_handle h = nullptr;
    // host arrays: every graph's vertices go to reverse Cuthill-McKee order,
    // so that a row's neighbours lie close to it and the products' gathers
    // share cache lines (the caller's ids of a geometric graph are unrelated
    // to its geometry); partition_batch maps its inputs and outputs back
    const bool reorder = !(flags & SPHYNX_DEVICE_PTRS);
    PermutedCsr P;
    if (reorder) {
      if (!row_ptr || !col || n < 1) fail(SPHYNX_ERR_INVALID_ARG, "NULL CSR array or empty batch");
      if (row_ptr[0] != 0 || row_ptr[n] != nnz) fail(SPHYNX_ERR_INVALID_ARG, "row_ptr must run from 0 to nnz");
      for (int64_t r = 0; r < n; ++r)
        if (row_ptr[r + 1] < row_ptr[r]) fail(SPHYNX_ERR_INVALID_ARG, "row_ptr decreases at row %lld",
                                                static_cast<long long>(r));
      for (int64_t k = 0; k < nnz; ++k)
        if (col[k] < 0 || col[k] >= n) fail(SPHYNX_ERR_INVALID_ARG, "column index out of range at entry %lld",
                                            static_cast<long long>(k));
      P = permute_batch(row_ptr, col, edge_w, vtx_w, graph_ptr, count, n);
    }
    const int rc = reorder ? sphynx_create(P.rp.data(), P.col.data(), edge_w ? P.w.data() : nullptr,
                                           vtx_w ? P.vw.data() : nullptr, n, nnz, flags, stream, &h)
                           : sphynx_create(row_ptr, col, edge_w, vtx_w, n, nnz, flags, stream, &h);
    if (rc != SPHYNX_OK) return rc;
    try {
      batch_setup(h, graph_ptr, count);
      if (reorder) {
        BatchInfo &B = h->batch;
        B.orig.alloc(static_cast<size_t>(n) * sizeof(int32_t));
        SPX_CUDA(cudaMemcpyAsync(B.orig.p, P.order.data(), static_cast<size_t>(n) * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, h->stream));
        if (vtx_w) {
          B.vw_orig.alloc(static_cast<size_t>(n) * sizeof(int64_t));
          SPX_CUDA(cudaMemcpyAsync(B.vw_orig.p, vtx_w, static_cast<size_t>(n) * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, h->stream));
        }
        SPX_CUDA(cudaStreamSynchronize(h->stream));   // the host arrays above go out of scope
      }
    } catch (...) {
      sphynx_destroy(h);
      throw;
    }
    *out = h;
    return SPHYNX_OK;
  });
}

extern "C" int sphynx_partition_batch(sphynx_handle g, int32_t K, const sphynx_options *opt, int32_t *part_out,
                                      double *cuts, double *imbalances, double *eigenvalues, int32_t *iterations,
                                      int32_t *status, sphynx_stats *stats) {
  return guarded([&]() -> int {
    if (!g || !part_out || !opt) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (g->batch.count < 1) fail(SPHYNX_ERR_INVALID_ARG, "the handle is not a batch (use sphynx_create_batch)");
    if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
    if (static_cast<int64_t>(K) * g->batch.count > (1 << 20)) fail(SPHYNX_ERR_UNSUPPORTED, "K x graphs > 2^20");
    check_lobpcg_options(g, opt);
    const auto t0 = std::chrono::steady_clock::now();
    const bool dev_out = (opt->flags & SPHYNX_OUT_DEVICE) != 0;
    int32_t *dpart = dev_out ? part_out
                             : static_cast<int32_t *>(g->workspace("part", static_cast<size_t>(g->n) * 4, false));
    if (stats) memset(stats, 0, sizeof(*stats));
    g->ctr.launches = 0;
    batch_partition(g, K, opt, dpart, cuts, imbalances, eigenvalues, iterations, status, stats);
    if (!dev_out)
      SPX_CUDA(cudaMemcpyAsync(part_out, dpart, static_cast<size_t>(g->n) * 4, cudaMemcpyDeviceToHost, g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    if (stats) {
      stats->kernel_launches = g->ctr.launches;
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return SPHYNX_OK;
  });
}
