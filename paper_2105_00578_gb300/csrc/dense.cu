// dense.cu -- the tall-skinny dense kernels of LOBPCG (Algorithm 1) and of the
// polynomial preconditioner's Lanczos setup (Sec. 5.2).
//
// Blocks are row-major n x ld (ld = 4, 8, 12 or 16).  Every kernel here reads
// and writes its blocks once with coalesced 16-byte accesses; reductions over
// n go through per-CTA partials in double that a second, fixed-order pass adds,
// so results do not depend on scheduling.
#include "internal.cuh"

#include <cmath>

namespace sphynx {

namespace {

template <typename T> __device__ inline T from_d(double v) { return static_cast<T>(v); }

// LD consecutive values (16-byte aligned) in 16-byte pieces
template <typename T, int LD>
__device__ __forceinline__ void row_load(const T *p, T (&o)[LD]) {
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int c = 0; c < LD; c += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(p + c);
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < LD; c += 2) {
      const double2 v = *reinterpret_cast<const double2 *>(p + c);
      o[c] = v.x; o[c + 1] = v.y;
    }
  }
}
template <typename T, int LD>
__device__ __forceinline__ void row_store(T *p, const T (&v)[LD]) {
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int c = 0; c < LD; c += 4) *reinterpret_cast<float4 *>(p + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < LD; c += 2) *reinterpret_cast<double2 *>(p + c) = make_double2(v[c], v[c + 1]);
  }
}

unsigned blocks_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1LL << 30)) b = (1LL << 30);
  return static_cast<unsigned>(b);
}

// ---------------------------------------------------------------------------
// initial blocks (Sec. 6.2.1)
template <typename T>
__global__ void k_random_block(T *x, int64_t n, int b, int ld, uint64_t state) {
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / ld;
    const int j = static_cast<int>(idx - i * ld);
    double v = 0.0;
    if (j < b) v = splitmix_pm1(state, static_cast<uint64_t>(i * b + j + 1));
    x[idx] = from_d<T>(v);
  }
}

template <typename T>
__global__ void k_piecewise_block(T *x, int64_t n, int b, int ld, int lap, const double *deg) {
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / ld;
    const int j = static_cast<int>(idx - i * ld);
    double v = 0.0;
    if (j == 0) {
      v = lap == SPHYNX_NORMALIZED ? sqrt(deg[i]) : 1.0;
    } else if (j < b) {
      const int64_t lo = (static_cast<int64_t>(j - 1) * n) / b, hi = (static_cast<int64_t>(j) * n) / b;
      v = (i >= lo && i < hi) ? 1.0 : 0.0;
    }
    x[idx] = from_d<T>(v);
  }
}

template <typename T>
__global__ void k_from_f64(T *x, const double *src, int64_t n, int b, int ld) {
  const int64_t total = n * ld;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / ld;
    const int j = static_cast<int>(idx - i * ld);
    x[idx] = from_d<T>(j < b ? src[i * b + j] : 0.0);
  }
}

template <typename T>
__global__ void k_to_f64(const T *x, double *dst, int64_t n, int b, int ld) {
  const int64_t total = n * b;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / b;
    const int j = static_cast<int>(idx - i * b);
    dst[idx] = static_cast<double>(x[i * ld + j]);
  }
}

// ---------------------------------------------------------------------------
// X' = S Y, P' = [0 H P] Y, LP' = [0 LH LP] Y  (Algorithm 1: the update and the new search directions)
template <typename T, int LD, int NBLK>
__global__ void __launch_bounds__(256)
k_update(int64_t n, const T *s0, const T *s1, const T *s2, const T *l1, const T *l2, const T *y,
         T *xo, T *po, T *lpo, const int *done) {
  constexpr int M = NBLK * LD;
  __shared__ __align__(16) T sy[M * LD];
  if (done && *done) return;
  for (int i = threadIdx.x; i < M * LD; i += blockDim.x) sy[i] = y[i];
  __syncthreads();
  const T *srows[3] = {s0, s1, s2};
  const T *lrows[3] = {nullptr, l1, l2};
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; row < n;
       row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    T x[LD], p[LD], lp[LD];
#pragma unroll
    for (int c = 0; c < LD; ++c) { x[c] = T(0); p[c] = T(0); lp[c] = T(0); }
#pragma unroll
    for (int blk = 0; blk < NBLK; ++blk) {
      // 4 columns of the input rows at a time; one coefficient row live at a time
#pragma unroll 1
      for (int k0 = 0; k0 < LD; k0 += 4) {
        T v[4], lv[4];
        row_load<T, 4>(srows[blk] + row * LD + k0, v);
        if (blk > 0) row_load<T, 4>(lrows[blk] + row * LD + k0, lv);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          T yr[LD];   // read once (a broadcast) for all three outputs
          row_load<T, LD>(sy + (blk * LD + k0 + kk) * LD, yr);
#pragma unroll
          for (int c = 0; c < LD; ++c) {
            x[c] += v[kk] * yr[c];
            if (blk > 0) {
              p[c] += v[kk] * yr[c];
              lp[c] += lv[kk] * yr[c];
            }
          }
        }
      }
    }
    row_store<T, LD>(xo + row * LD, x);
    if constexpr (NBLK == 3) {
      row_store<T, LD>(po + row * LD, p);
      row_store<T, LD>(lpo + row * LD, lp);
    }
  }
}

// ---------------------------------------------------------------------------
// R = L X - B X Theta (Algorithm 1: the residual), ||r_c||^2_{B^-1} partials, and
// the Jacobi scaling H = diag(L)^{-1} R (Sec. 5.1) when jinv is given.
template <typename T, int LD, typename TO = T>
__global__ void __launch_bounds__(256)
k_residual(int64_t n, const T *x, const T *lx, const double *theta, const T *bdiag, const T *jinv,
           TO *out, double *partials, const int *done) {
  __shared__ double red[256 / 32][LD];
  if (done && *done) return;
  T th[LD];
#pragma unroll
  for (int c = 0; c < LD; ++c) th[c] = static_cast<T>(theta[c]);
  T acc[LD];
#pragma unroll
  for (int c = 0; c < LD; ++c) acc[c] = T(0);
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; row < n;
       row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const T bi = bdiag ? bdiag[row] : T(1);
    const T ib = bdiag ? T(1) / bi : T(1);
    const T sc = jinv ? jinv[row] : T(1);
    T r[LD], xv[LD], lxv[LD];
    row_load<T, LD>(x + row * LD, xv);
    row_load<T, LD>(lx + row * LD, lxv);
#pragma unroll
    for (int c = 0; c < LD; ++c) {
      r[c] = lxv[c] - th[c] * (bi * xv[c]);
      acc[c] += r[c] * r[c] * ib;
      r[c] *= sc;
    }
    if constexpr (std::is_same<TO, __nv_bfloat16>::value) {
      // the norms above use the float residual; only the stored copy is rounded
#pragma unroll
      for (int c = 0; c < LD; c += 2)
        *reinterpret_cast<__nv_bfloat162 *>(out + row * LD + c) = __floats2bfloat162_rn(r[c], r[c + 1]);
    } else {
      row_store<T, LD>(out + row * LD, r);
    }
  }
  // block reduction in double, fixed order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < LD; ++c) {
    double v = static_cast<double>(acc[c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < LD) {
    double s = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    partials[static_cast<int64_t>(blockIdx.x) * LD + threadIdx.x] = s;
  }
}

// Convergence test (Algorithm 1, soft locking): ||r||_{B^-1} <= tol |theta|
// (abs_test: <= tol), or |theta| <= floor_th and ||r||_{B^-1} <= floor_res (the
// eigenvalue-zero vector).
__global__ void k_converge(SolverState *st, const double *partials, int grid, int b, int ld,
                           double tol, double floor_th, double floor_res, int count_iteration, int maxit,
                           int stall_window, int abs_test) {
  __shared__ double part[16][17];
  if (st->done) return;
  const int t = threadIdx.x;     // 256 threads: column t % 16, stripe t / 16
  const int c = t & 15, stripe = t >> 4;
  double s = 0.0;
  if (c < ld)
    for (int g = stripe; g < grid; g += 16) s += partials[static_cast<int64_t>(g) * ld + c];
  part[stripe][c] = s;
  __syncthreads();
  if (t == 0) {
    int nconv = 0;
    for (int j = 0; j < b; ++j) {
      double tot = 0.0;
      for (int q = 0; q < 16; ++q) tot += part[q][j];
      const double res = sqrt(tot);
      st->resnorm[j] = res;
      // the floor only admits the eigenvalue-zero vector (|theta| itself below it)
      const double th = fabs(st->theta[j]);
      const bool ok = (res <= (abs_test ? tol : tol * th)) || (th <= floor_th && res <= floor_res);
      st->conv[j] = ok ? 1 : 0;
      nconv += ok ? 1 : 0;
    }
    st->nconv = nconv;
    if (count_iteration) {
      st->iters += 1;
      st->pvalid = 1;
    }
    const bool stalled = stall_check(st, b, stall_window, count_iteration, floor_th);
    if (nconv == b) {
      st->done = 1;
      st->status = SPHYNX_OK;
    } else if (st->iters >= maxit || stalled) {
      st->done = 1;
      st->status = SPHYNX_ERR_NOCONV;
      st->stalled = stalled ? 1 : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// embedding signs: entry of largest magnitude of each column made positive
// (lowest row on ties), then coords[i][j] = sign_{j+1} X[i][j+1] (the
// embedding of Algorithm 2).
template <typename T>
__global__ void k_argmax_partial(const T *x, int64_t n, int ld, int b, double *pval, int64_t *pidx) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  for (int c = 0; c < b; ++c) {
    double best = -1.0, bestv = 0.0;
    int64_t bidx = INT64_MAX;
    for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; row < n;
         row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const double v = static_cast<double>(x[row * ld + c]);
      const double m = fabs(v);
      if (m > best) { best = m; bestv = v; bidx = row; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bidx;
    __shared__ double svv[256];
    svv[threadIdx.x] = bestv;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double a = sv[threadIdx.x], o = sv[threadIdx.x + s];
        const int64_t ia = si[threadIdx.x], io = si[threadIdx.x + s];
        if (o > a || (o == a && io < ia)) {
          sv[threadIdx.x] = o; si[threadIdx.x] = io; svv[threadIdx.x] = svv[threadIdx.x + s];
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      pval[(static_cast<int64_t>(blockIdx.x) * b + c) * 2] = sv[0];
      pval[(static_cast<int64_t>(blockIdx.x) * b + c) * 2 + 1] = svv[0];
      pidx[static_cast<int64_t>(blockIdx.x) * b + c] = si[0];
    }
    __syncthreads();
  }
}

__global__ void k_argmax_final(const double *pval, const int64_t *pidx, int grid, int b, double *sign) {
  const int c = threadIdx.x;
  if (c >= b) return;
  double best = -1.0, bestv = 0.0;
  int64_t bidx = INT64_MAX;
  for (int g = 0; g < grid; ++g) {
    const double m = pval[(static_cast<int64_t>(g) * b + c) * 2];
    const int64_t i = pidx[static_cast<int64_t>(g) * b + c];
    if (m > best || (m == best && i < bidx)) {
      best = m; bidx = i; bestv = pval[(static_cast<int64_t>(g) * b + c) * 2 + 1];
    }
  }
  sign[c] = bestv < 0.0 ? -1.0 : 1.0;
}

template <typename T>
__global__ void k_coords(const T *x, int64_t n, int ld, int b, const double *sign, T *coords) {
  const int dims = b - 1;
  const int64_t total = n * dims;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / dims;
    const int j = static_cast<int>(idx - i * dims);
    coords[idx] = sign[j + 1] < 0.0 ? -x[i * ld + j + 1] : x[i * ld + j + 1];
  }
}

// ---------------------------------------------------------------------------
// Lanczos helpers (Sec. 5.2 setup).  The basis V is column-major: column c
// starts at basis + c * ldv, with ldv a multiple of 4 so that every column is
// 16-byte aligned.  Threads take rows four at a time (one vector load per
// column); the n mod 4 tail rows go to the first threads of block 0.
__device__ __forceinline__ void ld4(const float *p, float (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
// coherent loads / stores for the vector a kernel updates in place
__device__ __forceinline__ void ld4_rw(const float *p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4_rw(const double *p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

constexpr int kLzCols = 8;   // basis columns per block of the dot-product kernel

// partials[block][c] = sum over the block's rows of V[:, c] . w, for the
// kLzCols columns c0 .. c0 + 7 (c < j1) of blockIdx.y; 256 threads per block.
template <typename T>
__global__ void __launch_bounds__(256)
k_lanczos_dots(const T *basis, int64_t ldv, int j1, const T *w, int64_t n, double *partials) {
  __shared__ double red[kLzCols][8];
  const int c0 = blockIdx.y * kLzCols;
  T acc[kLzCols];
#pragma unroll
  for (int c = 0; c < kLzCols; ++c) acc[c] = T(0);
  const int64_t nq = n >> 2;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < nq;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    T wv[4];
    ld4(w + 4 * q, wv);
#pragma unroll
    for (int c = 0; c < kLzCols; ++c) {
      if (c0 + c < j1) {
        T vv[4];
        ld4(basis + static_cast<int64_t>(c0 + c) * ldv + 4 * q, vv);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[c] = fma(vv[i], wv[i], acc[c]);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
    const int64_t r = (nq << 2) + threadIdx.x;
    const T wv = w[r];
#pragma unroll
    for (int c = 0; c < kLzCols; ++c)
      if (c0 + c < j1) acc[c] = fma(basis[static_cast<int64_t>(c0 + c) * ldv + r], wv, acc[c]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kLzCols; ++c) {
    double d = static_cast<double>(acc[c]);
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
    if (lane == 0) red[c][warp] = d;
  }
  __syncthreads();
  if (threadIdx.x < kLzCols && c0 + static_cast<int>(threadIdx.x) < j1) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[threadIdx.x][k];
    partials[static_cast<int64_t>(blockIdx.x) * j1 + c0 + threadIdx.x] = s;
  }
}

__global__ void k_reduce_cols(const double *partials, int grid, int cols, double *out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int g = threadIdx.x; g < grid; g += blockDim.x) s += partials[static_cast<int64_t>(g) * cols + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// w <- w - V[:, :j1] h, and npart[block] = the block's part of ||w||^2.
template <typename T>
__global__ void __launch_bounds__(256)
k_lanczos_sub(const T *basis, int64_t ldv, int j1, T *w, int64_t n, const double *h, double *npart) {
  __shared__ T sh[SPHYNX_MAX_POLY_DEGREE + 1];
  __shared__ double red[8];
  for (int c = threadIdx.x; c < j1; c += blockDim.x) sh[c] = static_cast<T>(h[c]);
  __syncthreads();
  T acc = 0;
  const int64_t nq = n >> 2;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < nq;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    T v[4];
    ld4_rw(w + 4 * q, v);
#pragma unroll 4
    for (int c = 0; c < j1; ++c) {
      T b[4];
      ld4(basis + static_cast<int64_t>(c) * ldv + 4 * q, b);
      const T hc = sh[c];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] -= b[i] * hc;
    }
    st4(w + 4 * q, v);
#pragma unroll
    for (int i = 0; i < 4; ++i) acc += v[i] * v[i];
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
    const int64_t r = (nq << 2) + threadIdx.x;
    T v = w[r];
    for (int c = 0; c < j1; ++c) v -= basis[static_cast<int64_t>(c) * ldv + r] * sh[c];
    w[r] = v;
    acc += v * v;
  }
  double d = static_cast<double>(acc);
  for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += red[k];
    npart[blockIdx.x] = s;
  }
}

// v = w / beta and V[:, j] = v
template <typename T>
__global__ void k_lanczos_next(const T *w, T *v, T *basis, int64_t ldv, int j, int64_t n, const double *beta2) {
  const T inv = static_cast<T>(1.0 / sqrt(*beta2));
  T *col = basis + static_cast<int64_t>(j) * ldv;
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; row < n;
       row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const T val = w[row] * inv;
    v[row] = val;
    col[row] = val;
  }
}

template <typename T>
__global__ void k_poly_start(T *v, int64_t n, uint64_t state) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[i] = static_cast<T>(splitmix_pm1(state, static_cast<uint64_t>(i + 1)));
}

// partials of z.v and z.z with z the null vector (1, or sqrt(deg) for L_N)
template <typename T>
__global__ void __launch_bounds__(256)
k_null_dots(const T *v, int64_t n, int lap, const double *deg, double *partials) {
  __shared__ double r0[8], r1[8];
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double z = lap == SPHYNX_NORMALIZED ? sqrt(deg[i]) : 1.0;
    a0 += z * static_cast<double>(v[i]);
    a1 += z * z;
  }
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, off);
    a1 += __shfl_down_sync(0xffffffffu, a1, off);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = a0; r1[threadIdx.x >> 5] = a1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < 8; ++k) { s0 += r0[k]; s1 += r1[k]; }
    partials[blockIdx.x * 2] = s0;
    partials[blockIdx.x * 2 + 1] = s1;
  }
}

template <typename T>
__global__ void k_null_axpy(T *v, int64_t n, int lap, const double *deg, const double *scal) {
  const double f = scal[0] / scal[1];
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double z = lap == SPHYNX_NORMALIZED ? sqrt(deg[i]) : 1.0;
    v[i] = static_cast<T>(static_cast<double>(v[i]) - f * z);
  }
}

// ---- canonical rotation of a cluster of eigenvectors (embedding) ----------
// Row p of M = E_c^T Z_c for the cluster columns a .. a + c - 1, with Z the
// seeded reference block (entry (i, j): draw i * d + j + 1 of the stream that
// starts at `state`): partials[block][q] = the block's part of
// sum_i E[i, a + p] Z[i, a + q], q < c.
template <typename T>
__global__ void __launch_bounds__(256)
k_cluster_dots(const T *x, int64_t n, int ld, int d, int a, int c, int p, uint64_t state, double *partials) {
  __shared__ double red[8][SPHYNX_MAX_NEV];
  double acc[SPHYNX_MAX_NEV];
#pragma unroll
  for (int q = 0; q < SPHYNX_MAX_NEV; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double xv = static_cast<double>(x[i * ld + a + p]);
    const uint64_t base = static_cast<uint64_t>(i) * d + a + 1;
#pragma unroll
    for (int q = 0; q < SPHYNX_MAX_NEV; ++q)
      if (q < c) acc[q] += xv * splitmix_pm1(state, base + q);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < SPHYNX_MAX_NEV; ++q) {
    if (q >= c) break;
    double v = acc[q];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < c) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    partials[static_cast<int64_t>(blockIdx.x) * c + threadIdx.x] = s;
  }
}

// E_c <- E_c Q (Q row-major c x c) for the cluster columns a .. a + c - 1
template <typename T>
__global__ void k_rotate_cols(T *x, int64_t n, int ld, int a, int c, const double *q) {
  __shared__ double sq[SPHYNX_MAX_NEV * SPHYNX_MAX_NEV];
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) sq[e] = q[e];
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double v[SPHYNX_MAX_NEV];
#pragma unroll
    for (int p = 0; p < SPHYNX_MAX_NEV; ++p)
      if (p < c) v[p] = static_cast<double>(x[i * ld + a + p]);
#pragma unroll
    for (int k = 0; k < SPHYNX_MAX_NEV; ++k) {
      if (k >= c) break;
      double y = 0.0;
      for (int p = 0; p < c; ++p) y += v[p] * sq[p * c + k];
      x[i * ld + a + k] = static_cast<T>(y);
    }
  }
}

// col = z / ||z|| with z the null vector (1, or sqrt(deg) for L_N); scal[1] = z . z
template <typename T>
__global__ void k_null_column(T *col, int64_t n, int lap, const double *deg, const double *scal) {
  const double f = 1.0 / sqrt(scal[1]);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double z = lap == SPHYNX_NORMALIZED ? sqrt(deg[i]) : 1.0;
    col[i] = static_cast<T>(z * f);
  }
}

// H = R / theta_1 (a polynomial of degree one)
template <typename T>
__global__ void k_poly_single(const T *r, T *h, int64_t total, const double *inv, const int *done) {
  if (done && *done) return;
  const T f = static_cast<T>(inv[0]);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    h[i] = r[i] * f;
}

}  // namespace

// ===========================================================================
// host launchers

int vec_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 4 * kSmCount) g = 4 * kSmCount;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

void launch_zero(cudaStream_t s, void *p, size_t bytes) {
  if (bytes) SPX_CUDA(cudaMemsetAsync(p, 0, bytes, s));
}

void launch_random_block(cudaStream_t s, DT dt, void *x, int64_t n, int b, int ld, uint64_t seed) {
  const uint64_t state = mix64(seed + kGamma);
  const unsigned g = blocks_for(n * ld, 256) > 8192 ? 8192 : blocks_for(n * ld, 256);
  if (dt == DT::F64) k_random_block<double><<<g, 256, 0, s>>>(static_cast<double *>(x), n, b, ld, state);
  else k_random_block<float><<<g, 256, 0, s>>>(static_cast<float *>(x), n, b, ld, state);
  SPX_LAUNCHED();
}

void launch_piecewise_block(cudaStream_t s, DT dt, void *x, int64_t n, int b, int ld, int lap,
                            const double *deg) {
  const unsigned g = blocks_for(n * ld, 256) > 8192 ? 8192 : blocks_for(n * ld, 256);
  if (dt == DT::F64) k_piecewise_block<double><<<g, 256, 0, s>>>(static_cast<double *>(x), n, b, ld, lap, deg);
  else k_piecewise_block<float><<<g, 256, 0, s>>>(static_cast<float *>(x), n, b, ld, lap, deg);
  SPX_LAUNCHED();
}

void launch_from_f64(cudaStream_t s, DT dt, void *x, const double *src, int64_t n, int b, int ld) {
  const unsigned g = blocks_for(n * ld, 256) > 8192 ? 8192 : blocks_for(n * ld, 256);
  if (dt == DT::F64) k_from_f64<double><<<g, 256, 0, s>>>(static_cast<double *>(x), src, n, b, ld);
  else k_from_f64<float><<<g, 256, 0, s>>>(static_cast<float *>(x), src, n, b, ld);
  SPX_LAUNCHED();
}

void launch_to_f64(cudaStream_t s, DT dt, const void *x, double *dst, int64_t n, int b, int ld) {
  const unsigned g = blocks_for(n * b, 256) > 8192 ? 8192 : blocks_for(n * b, 256);
  if (dt == DT::F64) k_to_f64<double><<<g, 256, 0, s>>>(static_cast<const double *>(x), dst, n, b, ld);
  else k_to_f64<float><<<g, 256, 0, s>>>(static_cast<const float *>(x), dst, n, b, ld);
  SPX_LAUNCHED();
}

template <typename T, int LD>
static void update_ld(cudaStream_t st, const UpdateArgs &a, unsigned g) {
  const T *s0 = static_cast<const T *>(a.s[0]);
  const T *y = static_cast<const T *>(a.y);
  if (a.nblk == 1) {
    k_update<T, LD, 1><<<g, 256, 0, st>>>(a.n, s0, nullptr, nullptr, nullptr, nullptr, y,
                                          static_cast<T *>(a.xo), nullptr, nullptr, a.done);
  } else {
    k_update<T, LD, 3><<<g, 256, 0, st>>>(
        a.n, s0, static_cast<const T *>(a.s[1]), static_cast<const T *>(a.s[2]),
        static_cast<const T *>(a.ls[1]), static_cast<const T *>(a.ls[2]), y, static_cast<T *>(a.xo),
        static_cast<T *>(a.po), static_cast<T *>(a.lpo), a.done);
  }
  SPX_LAUNCHED();
}

void launch_update(cudaStream_t st, const UpdateArgs &a) {
  if (a.nblk != 1 && a.nblk != 3) fail(SPHYNX_ERR_INVALID_ARG, "update: nblk %d", a.nblk);
  const unsigned g = static_cast<unsigned>(vec_grid(a.n) * 2);
  if (a.dt == DT::F64) {
    switch (a.ld) {
      case 4: update_ld<double, 4>(st, a, g); break;
      case 8: update_ld<double, 8>(st, a, g); break;
      case 12: update_ld<double, 12>(st, a, g); break;
      case 16: update_ld<double, 16>(st, a, g); break;
      default: fail(SPHYNX_ERR_INVALID_ARG, "update: ld %d", a.ld);
    }
  } else {
    switch (a.ld) {
      case 4: update_ld<float, 4>(st, a, g); break;
      case 8: update_ld<float, 8>(st, a, g); break;
      case 12: update_ld<float, 12>(st, a, g); break;
      case 16: update_ld<float, 16>(st, a, g); break;
      default: fail(SPHYNX_ERR_INVALID_ARG, "update: ld %d", a.ld);
    }
  }
}

int residual_grid(int64_t n) { return vec_grid(n); }

template <typename T, int LD>
static void residual_ld(cudaStream_t st, const ResidualArgs &a, int grid) {
  const T *bd = nullptr, *jv = nullptr;
  if constexpr (std::is_same<T, double>::value) {
    bd = a.bdiag;
    jv = a.jinv;
  } else {
    bd = a.bdiagf;
    jv = a.jinvf;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (a.out_bf16) {
      k_residual<float, LD, __nv_bfloat16><<<grid, 256, 0, st>>>(
          a.n, static_cast<const float *>(a.x), static_cast<const float *>(a.lx), a.theta, bd, jv,
          static_cast<__nv_bfloat16 *>(a.out), a.norm_partials, a.done);
      SPX_LAUNCHED();
      return;
    }
  }
  k_residual<T, LD><<<grid, 256, 0, st>>>(a.n, static_cast<const T *>(a.x), static_cast<const T *>(a.lx),
                                          a.theta, bd, jv, static_cast<T *>(a.out), a.norm_partials, a.done);
  SPX_LAUNCHED();
}

void launch_residual(cudaStream_t st, const ResidualArgs &a, int grid) {
  if (a.dt == DT::F64) {
    switch (a.ld) {
      case 4: residual_ld<double, 4>(st, a, grid); break;
      case 8: residual_ld<double, 8>(st, a, grid); break;
      case 12: residual_ld<double, 12>(st, a, grid); break;
      case 16: residual_ld<double, 16>(st, a, grid); break;
      default: fail(SPHYNX_ERR_INVALID_ARG, "residual: ld %d", a.ld);
    }
  } else {
    switch (a.ld) {
      case 4: residual_ld<float, 4>(st, a, grid); break;
      case 8: residual_ld<float, 8>(st, a, grid); break;
      case 12: residual_ld<float, 12>(st, a, grid); break;
      case 16: residual_ld<float, 16>(st, a, grid); break;
      default: fail(SPHYNX_ERR_INVALID_ARG, "residual: ld %d", a.ld);
    }
  }
}

void launch_converge(cudaStream_t st, SolverState *state, const double *partials, int grid, int b,
                     int ld, double tol, double floor_th, double floor_res, int count_iteration, int maxit,
                     int stall_window, int abs_test) {
  k_converge<<<1, 256, 0, st>>>(state, partials, grid, b, ld, tol, floor_th, floor_res, count_iteration, maxit,
                                stall_window, abs_test);
  SPX_LAUNCHED();
}

void launch_signs_coords(cudaStream_t st, DT dt, const void *x, int64_t n, int ld, int b,
                         void *coords, double *scratch) {
  const int grid = vec_grid(n);
  double *pval = scratch;                                            // grid * b * 2
  int64_t *pidx = reinterpret_cast<int64_t *>(scratch + static_cast<size_t>(grid) * b * 2);
  double *sign = scratch + static_cast<size_t>(grid) * b * 3;         // b
  if (dt == DT::F64) {
    k_argmax_partial<double><<<grid, 256, 0, st>>>(static_cast<const double *>(x), n, ld, b, pval, pidx);
  } else {
    k_argmax_partial<float><<<grid, 256, 0, st>>>(static_cast<const float *>(x), n, ld, b, pval, pidx);
  }
  SPX_LAUNCHED();
  k_argmax_final<<<1, 32, 0, st>>>(pval, pidx, grid, b, sign);
  SPX_LAUNCHED();
  if (b > 1) {
    const unsigned g = blocks_for(n * (b - 1), 256) > 8192 ? 8192 : blocks_for(n * (b - 1), 256);
    if (dt == DT::F64)
      k_coords<double><<<g, 256, 0, st>>>(static_cast<const double *>(x), n, ld, b, sign, static_cast<double *>(coords));
    else
      k_coords<float><<<g, 256, 0, st>>>(static_cast<const float *>(x), n, ld, b, sign, static_cast<float *>(coords));
    SPX_LAUNCHED();
  }
}

void launch_lanczos_dots(cudaStream_t st, DT dt, const void *basis, int64_t ldv, int j1, const void *w,
                         int64_t n, double *partials, int grid) {
  if (ldv % 4 || reinterpret_cast<uintptr_t>(basis) % 32 || reinterpret_cast<uintptr_t>(w) % 32)
    fail(SPHYNX_ERR_INVALID_ARG, "Lanczos basis columns must be 32-byte aligned");
  const dim3 g(static_cast<unsigned>(grid), static_cast<unsigned>((j1 + kLzCols - 1) / kLzCols));
  if (dt == DT::F64)
    k_lanczos_dots<double><<<g, 256, 0, st>>>(static_cast<const double *>(basis), ldv, j1,
                                              static_cast<const double *>(w), n, partials);
  else
    k_lanczos_dots<float><<<g, 256, 0, st>>>(static_cast<const float *>(basis), ldv, j1,
                                             static_cast<const float *>(w), n, partials);
  SPX_LAUNCHED();
}

void launch_reduce_cols(cudaStream_t st, const double *partials, int grid, int cols, double *out) {
  k_reduce_cols<<<cols, 256, 0, st>>>(partials, grid, cols, out);
  SPX_LAUNCHED();
}

void launch_lanczos_sub(cudaStream_t st, DT dt, const void *basis, int64_t ldv, int j1, void *w, int64_t n,
                        const double *h, double *norm_partials, int grid) {
  if (ldv % 4 || reinterpret_cast<uintptr_t>(basis) % 32 || reinterpret_cast<uintptr_t>(w) % 32)
    fail(SPHYNX_ERR_INVALID_ARG, "Lanczos basis columns must be 32-byte aligned");
  if (dt == DT::F64)
    k_lanczos_sub<double><<<grid, 256, 0, st>>>(static_cast<const double *>(basis), ldv, j1,
                                                static_cast<double *>(w), n, h, norm_partials);
  else
    k_lanczos_sub<float><<<grid, 256, 0, st>>>(static_cast<const float *>(basis), ldv, j1,
                                               static_cast<float *>(w), n, h, norm_partials);
  SPX_LAUNCHED();
}

void launch_lanczos_next(cudaStream_t st, DT dt, const void *w, void *v, void *basis, int64_t ldv, int j,
                         int64_t n, const double *beta2) {
  const int g = vec_grid(n);
  if (dt == DT::F64)
    k_lanczos_next<double><<<g, 256, 0, st>>>(static_cast<const double *>(w), static_cast<double *>(v),
                                              static_cast<double *>(basis), ldv, j, n, beta2);
  else
    k_lanczos_next<float><<<g, 256, 0, st>>>(static_cast<const float *>(w), static_cast<float *>(v),
                                             static_cast<float *>(basis), ldv, j, n, beta2);
  SPX_LAUNCHED();
}

void launch_poly_start(cudaStream_t st, DT dt, void *v, int64_t n, uint64_t seed) {
  const uint64_t state = mix64(seed + 3 * kGamma);
  const int g = vec_grid(n);
  if (dt == DT::F64) k_poly_start<double><<<g, 256, 0, st>>>(static_cast<double *>(v), n, state);
  else k_poly_start<float><<<g, 256, 0, st>>>(static_cast<float *>(v), n, state);
  SPX_LAUNCHED();
}

void launch_project_null(cudaStream_t st, DT dt, void *v, int64_t n, int lap, const double *deg,
                         double *partials, int grid, double *scal) {
  if (dt == DT::F64)
    k_null_dots<double><<<grid, 256, 0, st>>>(static_cast<const double *>(v), n, lap, deg, partials);
  else
    k_null_dots<float><<<grid, 256, 0, st>>>(static_cast<const float *>(v), n, lap, deg, partials);
  SPX_LAUNCHED();
  k_reduce_cols<<<2, 256, 0, st>>>(partials, grid, 2, scal);
  SPX_LAUNCHED();
  if (dt == DT::F64) k_null_axpy<double><<<grid, 256, 0, st>>>(static_cast<double *>(v), n, lap, deg, scal);
  else k_null_axpy<float><<<grid, 256, 0, st>>>(static_cast<float *>(v), n, lap, deg, scal);
  SPX_LAUNCHED();
}

void launch_cluster_dots(cudaStream_t st, DT dt, const void *x, int64_t n, int ld, int d, int a, int c, int p,
                         uint64_t seed, double *partials, int grid) {
  if (c < 1 || c > SPHYNX_MAX_NEV || a < 0 || a + c > ld || p < 0 || p >= c)
    fail(SPHYNX_ERR_INVALID_ARG, "cluster columns out of range");
  const uint64_t state = mix64(seed + 5 * kGamma);
  if (dt == DT::F64)
    k_cluster_dots<double><<<grid, 256, 0, st>>>(static_cast<const double *>(x), n, ld, d, a, c, p, state, partials);
  else
    k_cluster_dots<float><<<grid, 256, 0, st>>>(static_cast<const float *>(x), n, ld, d, a, c, p, state, partials);
  SPX_LAUNCHED();
}

void launch_rotate_cols(cudaStream_t st, DT dt, void *x, int64_t n, int ld, int a, int c, const double *q) {
  if (c < 1 || c > SPHYNX_MAX_NEV || a < 0 || a + c > ld) fail(SPHYNX_ERR_INVALID_ARG, "cluster columns out of range");
  const int g = vec_grid(n);
  if (dt == DT::F64) k_rotate_cols<double><<<g, 256, 0, st>>>(static_cast<double *>(x), n, ld, a, c, q);
  else k_rotate_cols<float><<<g, 256, 0, st>>>(static_cast<float *>(x), n, ld, a, c, q);
  SPX_LAUNCHED();
}

void launch_null_column(cudaStream_t st, DT dt, void *col, int64_t n, int lap, const double *deg,
                        const double *scal) {
  const int g = vec_grid(n);
  if (dt == DT::F64) k_null_column<double><<<g, 256, 0, st>>>(static_cast<double *>(col), n, lap, deg, scal);
  else k_null_column<float><<<g, 256, 0, st>>>(static_cast<float *>(col), n, lap, deg, scal);
  SPX_LAUNCHED();
}

void launch_poly_single(cudaStream_t st, DT dt, const void *r, void *h, int64_t n, int ld,
                        const double *inv, const int *done) {
  const int g = vec_grid(n * ld);
  if (dt == DT::F64)
    k_poly_single<double><<<g, 256, 0, st>>>(static_cast<const double *>(r), static_cast<double *>(h), n * ld, inv, done);
  else
    k_poly_single<float><<<g, 256, 0, st>>>(static_cast<const float *>(r), static_cast<float *>(h), n * ld, inv, done);
  SPX_LAUNCHED();
}

}  // namespace sphynx

namespace sphynx {
namespace {
__global__ void k_d2f(const double *src, float *dst, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[i] = static_cast<float>(src[i]);
}
}  // namespace
void launch_d2f(cudaStream_t st, const double *src, float *dst, int64_t n) {
  k_d2f<<<vec_grid(n), 256, 0, st>>>(src, dst, n);
  SPX_LAUNCHED();
}
}  // namespace sphynx
