// small.cu -- FP64 small dense algebra on the GPU, one CTA per problem.
//
// * Rayleigh-Ritz (Sec. 3.3; the Rayleigh-Ritz steps of Algorithm 1): with G_A = S^T L S
//   and G_B = S^T B S restricted to the active columns of S and symmetrised,
//   scale to unit diagonal (D), factor D G_B D = R^T R (Cholesky, the small
//   half of Cholesky-QR) and take C = R^{-1}; if a pivot falls below
//   tau = 10 m u_work, use the eigendecomposition D G_B D = U Lambda U^T
//   instead and keep the directions with lambda > tau lambda_max (SVQB).
//   Then solve C^T (D G_A D) C w = theta w and return the nev smallest
//   theta with Y = D C W (each w signed so its largest entry is positive).
// * Gram partial reduction: the per-CTA partials of the Gram kernel are added
//   in a fixed order, 8 threads per entry.
// * Harmonic Ritz values (Sec. 5.2 setup): eigenvalues of
//   (T^2 + beta_k^2 e_k e_k^T) y = theta T y through T = R^T R, Leja ordered.
//
// The symmetric eigensolver is the cyclic Jacobi method with round-robin
// pairing (Golub and Van Loan, Matrix Computations, Sec. 8.5): m/2 disjoint
// rotations per round are applied by all threads at once (one 2 x 2 block of
// J^T A J per thread), rotations are skipped when
// |a_pq| <= 1e-15 (|a_pp| + |a_qq|), and sweeps stop when none was applied.
#include "internal.cuh"

#include <cfloat>
#include <climits>
#include <cmath>

namespace sphynx {

namespace {

constexpr int kMaxM = 3 * SPHYNX_MAX_NEV;   // 48
constexpr int kSmallThreads = 256;

// ---- cooperative building blocks (all threads of the CTA call them) --------

// In-place Cholesky of the leading m x m of B (ld): on success the upper
// triangle holds R with B = R^T R.  Returns the smallest pivot (R_kk^2) or
// a negative value if a pivot was not positive.
__device__ double chol_upper(double *B, int ld, int m, double *scratch) {
  const int tid = threadIdx.x;
  if (tid == 0) scratch[0] = INFINITY;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      const double d = B[k * ld + k];
      if (!(d > 0.0)) {
        scratch[0] = -1.0;
      } else {
        if (d < scratch[0]) scratch[0] = d;
        const double r = rsqrt(d);   // 1 / R_kk; R_kk = d r (the row below is scaled by r, not divided)
        B[k * ld + k] = d * r;
        scratch[1] = r;
      }
    }
    __syncthreads();
    if (scratch[0] < 0.0) return -1.0;
    const double rinv = scratch[1];
    for (int j = k + 1 + tid; j < m; j += blockDim.x) B[k * ld + j] *= rinv;
    __syncthreads();
    const int rem = m - k - 1;
    for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
      const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j >= i) B[i * ld + j] -= B[k * ld + i] * B[k * ld + j];
    }
    __syncthreads();
  }
  const double mn = scratch[0];
  __syncthreads();
  return mn;
}

// C = R^{-1} for upper-triangular R (leading m x m, ld); C is upper triangular.
// Thread j solves column j by back substitution; the pivot reciprocals are
// formed first, in parallel, so that no division sits on the column's
// dependent chain, and each dot product runs in two independent halves.
__device__ void tri_inv_upper(const double *R, int ld, int m, double *C, int ldc, double *rinv) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) C[(idx / m) * ldc + idx % m] = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) rinv[j] = 1.0 / R[j * ld + j];
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    C[j * ldc + j] = rinv[j];
    for (int i = j - 1; i >= 0; --i) {
      double s0 = 0.0, s1 = 0.0;
      int k = i + 1;
      for (; k + 1 <= j; k += 2) {
        s0 += R[i * ld + k] * C[k * ldc + j];
        s1 += R[i * ld + k + 1] * C[(k + 1) * ldc + j];
      }
      if (k <= j) s0 += R[i * ld + k] * C[k * ldc + j];
      C[i * ldc + j] = -(s0 + s1) * rinv[i];
    }
  }
  __syncthreads();
}

// Out (ra x cb) = op(A) (ra x ka) * Bm (ka x cb); transA reads A as its transpose.
__device__ void matmul(const double *A, int lda, bool transA, const double *Bm, int ldb, double *Out,
                       int ldo, int ra, int ka, int cb) {
  for (int idx = threadIdx.x; idx < ra * cb; idx += blockDim.x) {
    const int i = idx / cb, j = idx % cb;
    double s = 0.0;
    for (int k = 0; k < ka; ++k) s += (transA ? A[k * lda + i] : A[i * lda + k]) * Bm[k * ldb + j];
    Out[i * ldo + j] = s;
  }
  __syncthreads();
}

__device__ void symmetrize(double *A, int ld, int m) {
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    if (i < j) {
      const double v = 0.5 * (A[i * ld + j] + A[j * ld + i]);
      A[i * ld + j] = v;
      A[j * ld + i] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double inv_sqrt(double v) { return rsqrt(v); }
__device__ __forceinline__ float inv_sqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double abs_t(double v) { return fabs(v); }
__device__ __forceinline__ float abs_t(float v) { return fabsf(v); }

// Cyclic Jacobi: A (m x m, ld) -> diagonal of eigenvalues, V (ld) eigenvectors
// in columns, in double or float.  `cs` needs 2 * kMaxM entries of T, `pq`
// 2 * kMaxM ints.  A rotation is skipped below rel * (|a_pp| + |a_qq|), rel a
// few units of the type's rounding.  A round is two block barriers: the first
// (__syncthreads_count) publishes the rotations and counts them, the second
// ends their application.  The rounds' critical path is the rotation angle,
// so everything else is hoisted out of it: a thread decodes its share of the
// update once per call, and the round-robin partners advance by one with a
// wrap instead of a modulo.  In float the angle uses the fast reciprocal and
// reciprocal square root, whose rounding only perturbs the angle:
// c = rsqrt(1 + t^2), s = t c keep the rotation orthogonal to working accuracy.
__device__ __forceinline__ double jrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float jrcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double jsqrt1(double x) { return sqrt(x); }
__device__ __forceinline__ float jsqrt1(float x) { return x * rsqrtf(x); }   // x >= 1

// update items per thread: np^2 blocks of A plus m np entries of V, at most
// 24 * 24 + 48 * 24 = 1728 for m = kMaxM, over kSmallThreads threads
constexpr int kJacobiItems = (24 * 24 + 48 * 24 + 255) / 256;
static_assert(kMaxM == 48 && kSmallThreads == 256, "kJacobiItems assumes m <= 48 and 256 threads");

template <typename T>
__device__ void jacobi_eig(T *A, int ld, T *V, int ldv, int m, T *cs, int *pq) {
  const T rel = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    V[i * ldv + j] = i == j ? T(1) : T(0);
  }
  __syncthreads();
  if (m < 2) return;
  const int mp = m + (m & 1);
  const int np = mp / 2;
  // this thread's update items: 2 x 2 blocks (k, l) of A, then entries (i, l) of V
  int ik[kJacobiItems], il[kJacobiItems];
  int nitems = 0;
#pragma unroll
  for (int u = 0; u < kJacobiItems; ++u) {
    const int idx = tid + u * static_cast<int>(blockDim.x);
    ik[u] = -1;
    il[u] = 0;
    if (idx < np * np) {
      ik[u] = idx / np;
      il[u] = idx - (idx / np) * np;
      nitems = u + 1;
    } else if (idx < np * np + m * np) {
      const int it = idx - np * np;
      ik[u] = np + it / np;   // >= np marks a V row: i = ik - np
      il[u] = it - (it / np) * np;
      nitems = u + 1;
    }
  }
  // round-robin partners of pair k (thread k < np): position 0 stays, the
  // others cycle through 1 .. mp - 1
  const int k2 = mp - 1 - tid;
  for (int sweep = 0; sweep < 40; ++sweep) {
    int rotations = 0;   // the same in every thread: a sum of block-wide counts
    int a0 = tid == 0 ? 0 : ((tid - 1) % (mp - 1)) + 1;
    int a1 = tid < np ? ((k2 - 1) % (mp - 1)) + 1 : 0;
    for (int r = 0; r < mp - 1; ++r) {
      int rot = 0;
      if (tid < np) {
        const int p = a0 < a1 ? a0 : a1, q = a0 < a1 ? a1 : a0;
        T c = T(1), s = T(0);
        if (q < m) {
          const T app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
          if (apq != T(0) && abs_t(apq) > rel * (abs_t(app) + abs_t(aqq))) {
            const T tau = (aqq - app) * T(0.5) * jrcp(apq);
            const T t = tau == T(0) ? T(1)
                                    : (tau > T(0) ? T(1) : T(-1)) * jrcp(abs_t(tau) + jsqrt1(T(1) + tau * tau));
            c = inv_sqrt(T(1) + t * t);
            s = t * c;
            rot = 1;
          }
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        pq[2 * tid] = p;
        pq[2 * tid + 1] = q;
        if (tid != 0) a0 = a0 == mp - 1 ? 1 : a0 + 1;
        a1 = a1 == mp - 1 ? 1 : a1 + 1;
      }
      const int nrot = __syncthreads_count(rot);
      rotations += nrot;
      // A <- J^T A J one 2 x 2 block per pair of rotation pairs (the pairs are
      // disjoint, so the blocks are too), and V <- V J
      if (nrot) {
#pragma unroll
        for (int u = 0; u < kJacobiItems; ++u) {
          if (u >= nitems) break;
          const int k = ik[u], l = il[u];
          if (k < np) {
            const T ck = cs[2 * k], sk = cs[2 * k + 1];
            const T cl = cs[2 * l], sl = cs[2 * l + 1];
            if (sk == T(0) && sl == T(0)) continue;
            const int pk = pq[2 * k], qk = pq[2 * k + 1];
            const int pl = pq[2 * l], ql = pq[2 * l + 1];
            const bool hk = qk < m, hl = ql < m;
            const T a = A[pk * ld + pl];
            const T b = hl ? A[pk * ld + ql] : T(0);
            const T c = hk ? A[qk * ld + pl] : T(0);
            const T d = (hk && hl) ? A[qk * ld + ql] : T(0);
            // rows (J_k^T), then columns (J_l)
            const T r0a = ck * a - sk * c, r0b = ck * b - sk * d;
            const T r1a = sk * a + ck * c, r1b = sk * b + ck * d;
            A[pk * ld + pl] = cl * r0a - sl * r0b;
            if (hl) A[pk * ld + ql] = (k == l) ? T(0) : sl * r0a + cl * r0b;
            if (hk) A[qk * ld + pl] = (k == l) ? T(0) : cl * r1a - sl * r1b;
            if (hk && hl) A[qk * ld + ql] = sl * r1a + cl * r1b;
          } else if (k >= np) {
            const int i = k - np;
            const T cl = cs[2 * l], sl = cs[2 * l + 1];
            const int pl = pq[2 * l], ql = pq[2 * l + 1];
            if (sl == T(0) || ql >= m) continue;
            const T vp = V[i * ldv + pl], vq = V[i * ldv + ql];
            V[i * ldv + pl] = cl * vp - sl * vq;
            V[i * ldv + ql] = sl * vp + cl * vq;
          }
        }
      }
      __syncthreads();
    }
    if (rotations == 0) break;   // uniform: every thread summed the same counts
  }
}

// order[0..m) = indices of diag(A) sorted ascending (stable on equal values)
template <typename T>
__device__ void sort_diag(const T *A, int ld, int m, int *order) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const T di = A[i * ld + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const T dj = A[j * ld + j];
      if (dj < di || (dj == di && j < i)) ++rank;
    }
    order[rank] = i;
  }
  __syncthreads();
}

struct RRSmem {
  double A[kMaxM * kMaxM];   // scaled G_A (active)
  double B[kMaxM * kMaxM];   // scaled G_B -> R or U
  double C[kMaxM * kMaxM];   // basis coefficients C (m x m2)
  double T[kMaxM * kMaxM];   // temp
  double W[kMaxM * kMaxM];   // projected matrix -> eigenvalues on diagonal
  double V[kMaxM * kMaxM];   // eigenvectors of W
  double Bh[kMaxM * kMaxM];  // scaled G_B, kept for the Rayleigh quotients
  double P0[kMaxM * kMaxM];  // eigensolver workspaces of the float-started solve
  double P1[kMaxM * kMaxM];
  double P2[kMaxM * kMaxM];
  float A32[kMaxM * (kMaxM + 1)];  // float copies for the float-started solve (odd leading dimension)
  float V32[kMaxM * (kMaxM + 1)];
  float cs32[2 * kMaxM];
  int pq32[2 * kMaxM];
  double d[kMaxM];
  double rinv[kMaxM];        // reciprocal Cholesky pivots
  double cs[2 * kMaxM];      // Jacobi rotations (c, s) and pairs (p, q)
  int pq[2 * kMaxM];
  double qa[SPHYNX_MAX_NEV], qb[SPHYNX_MAX_NEV];
  double scratch[4];
  int idx[kMaxM];            // active column -> full index
  int order[kMaxM];
  int keep[kMaxM];
  int sel[SPHYNX_MAX_NEV];
  unsigned amask[2];         // active columns, one ballot per warp
  int m, m2, fail, svqb;
};

// Symmetric eigendecomposition of the leading m x m of A (ld kMaxM) into
// its diagonal and V, to FP64 accuracy.  Plain: cyclic Jacobi in double from
// the identity.  Float-started: cyclic Jacobi in float first gives a basis V0
// accurate to about 1e-7; V0 is made orthonormal in double (Cholesky-QR: V0
// R^{-1} with V0^T V0 = R^T R), A1 = V0^T A V0 is then diagonal up to about
// 1e-7 |A|, and double Jacobi from there (quadratic convergence: two or three
// sweeps instead of seven or eight from the identity) finishes it: V = V0 V1.
// The result is the double solve's, only its starting basis comes from float
// arithmetic; on GB300, whose FP64 rate is 1/64 of FP32's, that halves the
// Rayleigh-Ritz step.
__device__ void eig_sym(RRSmem &S, double *A, double *V, int m, bool float_start) {
  const int L = kMaxM;
  if (!float_start || m < 2) {
    jacobi_eig<double>(A, L, V, L, m, S.cs, S.pq);
    return;
  }
  constexpr int L32 = kMaxM + 1;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    S.A32[(e / m) * L32 + e % m] = static_cast<float>(A[(e / m) * L + e % m]);
  __syncthreads();
  jacobi_eig<float>(S.A32, L32, S.V32, L32, m, S.cs32, S.pq32);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    S.P0[i * L + j] = static_cast<double>(S.V32[i * L32 + j]);
  }
  __syncthreads();
  matmul(S.P0, L, true, S.P0, L, S.P1, L, m, m, m);                 // G = V0^T V0
  if (chol_upper(S.P1, L, m, S.scratch) <= 0.0) {                   // G = R^T R (never fails near I)
    jacobi_eig<double>(A, L, V, L, m, S.cs, S.pq);
    return;
  }
  tri_inv_upper(S.P1, L, m, S.P2, L, S.rinv);                       // R^{-1}
  matmul(S.P0, L, false, S.P2, L, S.P1, L, m, m, m);                // V0 <- V0 R^{-1}, orthonormal
  matmul(A, L, false, S.P1, L, S.P2, L, m, m, m);                   // A V0
  matmul(S.P1, L, true, S.P2, L, S.P0, L, m, m, m);                 // A1 = V0^T A V0
  symmetrize(S.P0, L, m);
  jacobi_eig<double>(S.P0, L, S.P2, L, m, S.cs, S.pq);              // A1 = V1 diag V1^T
  matmul(S.P1, L, false, S.P2, L, V, L, m, m, m);                   // V = V0 V1
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    A[i * L + j] = i == j ? S.P0[i * L + i] : 0.0;
  }
  __syncthreads();
}

// One Rayleigh-Ritz step.  ga/gb: full M x M (device).  The active mask is
// taken from `active` (if not NULL) or derived from the solver state.
__global__ void __launch_bounds__(kSmallThreads)
k_rayleigh_ritz(const double *ga, const double *gb, int M, int ld, int nev, double u_work,
                SolverState *st, const int *active, double *y64, void *yt, int yt_f32,
                double *theta_out, int *svqb_out, int mixed) {
  extern __shared__ __align__(16) unsigned char smraw[];
  RRSmem &S = *reinterpret_cast<RRSmem *>(smraw);
  const int tid = threadIdx.x;
  // a launch of several CTAs solves that many problems laid out back to back
  // (a batch of graphs): CTA bi takes the bi-th of every array
  if (blockIdx.x > 0) {
    const size_t bi = blockIdx.x;
    ga += bi * M * M;
    gb += bi * M * M;
    if (st) st += bi;
    if (active) active += bi * M;
    if (y64) y64 += bi * M * ld;
    if (yt) yt = static_cast<char *>(yt) + bi * M * ld * (yt_f32 ? 4 : 8);
    if (theta_out) theta_out += bi * nev;
    if (svqb_out) svqb_out += bi;
  }
  if (st && st->done) return;
  const int L = kMaxM;  // leading dimension of the shared matrices
  // active columns: thread k < M tests column k, two warp ballots compact them
  if (tid < 64) {
    const int k = tid;
    bool a = false;
    if (k < M) {
      if (active) {
        a = active[k] != 0;
      } else {
        const int blk = k / ld, c = k % ld;
        a = c < nev && (blk == 0 || (!st->conv[c] && (blk == 1 || st->pvalid)));
      }
      const double dg = gb[k * M + k];
      a = a && isfinite(dg) && dg > 0.0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, a);
    if ((tid & 31) == 0) S.amask[tid >> 5] = bal;
  }
  if (tid == 0) {
    S.fail = 0;
    S.svqb = 0;
  }
  __syncthreads();
  if (tid < 64) {
    const unsigned m0 = S.amask[0], mine = tid < 32 ? m0 : S.amask[1];
    const int lane = tid & 31;
    if ((mine >> lane) & 1u) S.idx[(tid < 32 ? 0 : __popc(m0)) + __popc(mine & ((1u << lane) - 1u))] = tid;
    if (tid == 0) S.m = __popc(m0) + __popc(S.amask[1]);
  }
  __syncthreads();
  const int m = S.m;
  for (int i = tid; i < m; i += blockDim.x) S.d[i] = 1.0 / sqrt(gb[S.idx[i] * M + S.idx[i]]);
  __syncthreads();
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    const int fi = S.idx[i], fj = S.idx[j];
    const double di = S.d[i], dj = S.d[j];
    S.A[i * L + j] = 0.5 * (ga[fi * M + fj] + ga[fj * M + fi]) * di * dj;
    S.B[i * L + j] = 0.5 * (gb[fi * M + fj] + gb[fj * M + fi]) * di * dj;
  }
  __syncthreads();
  const double tau = 10.0 * m * u_work;
  // keep copies of the scaled G_B: for the SVQB fallback (T) and the final
  // Rayleigh quotients (Bh)
  for (int e = tid; e < m * m; e += blockDim.x) {
    S.T[(e / m) * L + e % m] = S.B[(e / m) * L + e % m];
    S.Bh[(e / m) * L + e % m] = S.B[(e / m) * L + e % m];
  }
  __syncthreads();
  const double minpiv = chol_upper(S.B, L, m, S.scratch);
  int m2 = m;
  if (minpiv >= tau) {
    tri_inv_upper(S.B, L, m, S.C, L, S.rinv);
  } else {
    // SVQB: eigendecomposition of the scaled G_B (copy in T)
    if (tid == 0) S.svqb = 1;
    eig_sym(S, S.T, S.V, m, mixed != 0);
    if (tid == 0) {
      double lmax = 0.0;
      for (int i = 0; i < m; ++i) lmax = fmax(lmax, S.T[i * L + i]);
      int c = 0;
      for (int i = 0; i < m; ++i)
        if (S.T[i * L + i] > tau * lmax) S.keep[c++] = i;
      S.m2 = c;
    }
    __syncthreads();
    m2 = S.m2;
    for (int e = tid; e < m * m2; e += blockDim.x) {
      const int i = e / m2, j = e % m2;
      const int kj = S.keep[j];
      S.C[i * L + j] = S.V[i * L + kj] / sqrt(S.T[kj * L + kj]);
    }
    __syncthreads();
  }
  if (tid == 0) S.m2 = m2;
  // W = C^T A C
  matmul(S.A, L, false, S.C, L, S.T, L, m, m, m2);
  matmul(S.C, L, true, S.T, L, S.W, L, m2, m, m2);
  symmetrize(S.W, L, m2);
  eig_sym(S, S.W, S.V, m2, mixed != 0);
  sort_diag(S.W, L, m2, S.order);
  if (tid == 0 && m2 < nev) S.fail = 1;
  __syncthreads();
  if (S.fail) {
    if (tid == 0 && st) {
      st->done = 1;
      st->status = SPHYNX_ERR_BREAKDOWN;
    }
    if (tid == 0 && svqb_out) *svqb_out = -1;
    return;
  }
  // sign of each selected eigenvector: largest |entry| positive, first on ties
  if (tid < nev) {
    const int col = S.order[tid];
    double best = -1.0;
    int bi = 0;
    for (int k = 0; k < m2; ++k) {
      const double a = fabs(S.V[k * L + col]);
      if (a > best) { best = a; bi = k; }
    }
    S.keep[tid] = S.V[bi * L + col] < 0.0 ? -1 : 1;
  }
  __syncthreads();
  // y_c = C w_c in the scaled coordinates (m x nev)
  for (int e = tid; e < m * nev; e += blockDim.x) {
    const int i = e / nev, c = e % nev;
    const int col = S.order[c];
    double s = 0.0;
    for (int k = 0; k < m2; ++k) s += S.C[i * L + k] * S.V[k * L + col];
    S.T[i * L + c] = s * S.keep[c];
  }
  if (tid < nev) {
    S.sel[tid] = tid;
    S.qa[tid] = S.W[S.order[tid] * L + S.order[tid]];
    S.qb[tid] = 1.0;
  }
  __syncthreads();
  for (int e = tid; e < M * ld; e += blockDim.x) {
    if (y64) y64[e] = 0.0;
    if (yt) {
      if (yt_f32) static_cast<float *>(yt)[e] = 0.f;
      else static_cast<double *>(yt)[e] = 0.0;
    }
  }
  __syncthreads();
  // Y = D y (rows of inactive columns stay zero)
  for (int e = tid; e < m * nev; e += blockDim.x) {
    const int i = e / nev, c = e % nev;
    const int src = S.sel[c];
    const double v = S.d[i] * S.T[i * L + src];
    const int o = S.idx[i] * ld + c;
    if (y64) y64[o] = v;
    if (yt) {
      if (yt_f32) static_cast<float *>(yt)[o] = static_cast<float>(v);
      else static_cast<double *>(yt)[o] = v;
    }
  }
  if (tid < nev) {
    const double th = S.qa[S.sel[tid]];
    if (st) st->theta[tid] = th;
    if (theta_out) theta_out[tid] = th;
  }
  if (tid == 0) {
    if (st) st->svqb_steps += S.svqb;
    if (svqb_out) *svqb_out = S.svqb;
  }
}

// Harmonic Ritz values of the Lanczos tridiagonal T (Sec. 5.2 setup): the
// eigenvalues theta of (T^2 + beta^2 e e^T) y = theta T y, e the last unit
// vector.  With the Cholesky factor T = R^T R (R upper bidiagonal, diagonal r,
// superdiagonal s) and y = R^{-1} z this is the standard problem
//   Z z = theta z,  Z = R R^T + (beta^2 / r_{k-1}^2) e e^T,
// because R^{-T} T^2 R^{-1} = R R^T and R^{-T} e = e / r_{k-1}.  Z is symmetric
// tridiagonal: diagonal r_i^2 + s_i^2 (plus the rank-one term on the last
// entry), off-diagonal s_i r_{i+1}.
//
// Its eigenvalues come from Sturm sequence counts (Barth, Martin and
// Wilkinson, 1967) by multisection: one CTA of one warp per eigenvalue (so the
// FP64 work, which is scarce per SM on this part, spreads over k SMs), whose
// 32 lanes count at 32 interior points of the current bracket, narrowing it
// 33-fold per round.  The count uses the division-free three-term recurrence
// of the leading principal minors, p_i = (d_i - sigma) p_{i-1} - e_{i-1}^2 p_{i-2},
// whose sign changes number the eigenvalues below sigma; pairs (p_i, p_{i-1})
// are rescaled by exact powers of two to stay in range.  A second, single-CTA
// kernel puts the values in modified Leja order.

// number of eigenvalues of the tridiagonal (d, e2) smaller than sigma
__device__ int sturm_count(const double *d, const double *e2, int k, double sigma) {
  double pm2 = 0.0, pm1 = 1.0;
  int cnt = 0;
  for (int i = 0; i < k; ++i) {
    double p = (d[i] - sigma) * pm1;
    if (i > 0) p -= e2[i - 1] * pm2;
    if (p == 0.0) p = pm1 > 0.0 ? -0x1p-900 : 0x1p-900;   // a zero minor counts as a sign change
    if ((p < 0.0) != (pm1 < 0.0)) ++cnt;
    const double a = fmax(fabs(p), fabs(pm1));
    if (a > 0x1p500) {
      p *= 0x1p-500;
      pm1 *= 0x1p-500;
    } else if (a < 0x1p-500) {
      p *= 0x1p500;
      pm1 *= 0x1p500;
    }
    pm2 = pm1;
    pm1 = p;
  }
  return cnt;
}

// CTA i (32 threads): theta[i], the i-th smallest eigenvalue of Z.  Problem
// blockIdx.y of a batch reads and writes its arrays `stride` further on.
__global__ void __launch_bounds__(32)
k_harmonic_eig(const double *alpha, const double *beta2, int k, double *theta, int *err, int stride) {
  __shared__ double d[SPHYNX_MAX_POLY_DEGREE], e2[SPHYNX_MAX_POLY_DEGREE];
  __shared__ double glo, ghi;
  __shared__ int bad;
  const int lane = threadIdx.x, i = blockIdx.x;
  alpha += static_cast<int64_t>(blockIdx.y) * stride;
  beta2 += static_cast<int64_t>(blockIdx.y) * stride;
  theta += static_cast<int64_t>(blockIdx.y) * stride;
  err += blockIdx.y;
  if (lane == 0) {
    // T = R^T R: r_0 = sqrt(alpha_0), s_j = b_j / r_j, r_{j+1} = sqrt(alpha_{j+1} - s_j^2)
    double r[SPHYNX_MAX_POLY_DEGREE], sd[SPHYNX_MAX_POLY_DEGREE];
    int b = 0;
    for (int j = 0; j < k; ++j) {
      const double piv = alpha[j] - (j > 0 ? sd[j - 1] * sd[j - 1] : 0.0);
      if (!(piv > 0.0) || !isfinite(piv)) {
        b = 1;
        break;
      }
      r[j] = sqrt(piv);
      sd[j] = j + 1 < k ? sqrt(beta2[j]) / r[j] : 0.0;
    }
    bad = b;
    if (!b) {
      for (int j = 0; j < k; ++j) {
        d[j] = r[j] * r[j] + sd[j] * sd[j];
        if (j + 1 < k) {
          const double off = sd[j] * r[j + 1];
          e2[j] = off * off;
        }
      }
      d[k - 1] += beta2[k - 1] / (r[k - 1] * r[k - 1]);
      // Gershgorin interval, widened by a few units of roundoff
      double lo = INFINITY, hi = -INFINITY;
      for (int j = 0; j < k; ++j) {
        const double rad = (j > 0 ? sqrt(e2[j - 1]) : 0.0) + (j + 1 < k ? sqrt(e2[j]) : 0.0);
        lo = fmin(lo, d[j] - rad);
        hi = fmax(hi, d[j] + rad);
      }
      const double span = fmax(fabs(lo), fabs(hi));
      glo = lo - 4.0 * DBL_EPSILON * span;
      ghi = hi + 4.0 * DBL_EPSILON * span;
    }
  }
  __syncwarp();
  if (bad) {
    if (lane == 0) *err = 1;
    return;
  }
  // count(sigma) > i  <=>  sigma > theta_i
  double lo = glo, hi = ghi;
  for (int round = 0; round < 48; ++round) {
    const double w = hi - lo;
    if (!(w > 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)))) break;
    const double sig = lo + w * (static_cast<double>(lane + 1) / 33.0);
    const bool above = sig > lo && sig < hi ? sturm_count(d, e2, k, sig) > i : sig >= hi;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    const int j = m ? __ffs(m) - 1 : 32;             // first point above theta_i
    const double nlo = j == 0 ? lo : __shfl_sync(0xffffffffu, sig, j - 1);
    const double nhi = j == 32 ? hi : __shfl_sync(0xffffffffu, sig, j < 32 ? j : 31);
    if (!(nhi - nlo < w)) break;                      // no progress left at this precision
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) theta[i] = 0.5 * (lo + hi);
}

// Definiteness (Sec. 5.2 with Algorithm 1, which takes a positive definite
// preconditioner): p(lambda) = (1 - prod_i (1 - lambda/theta_i)) / lambda is
// evaluated on lambda_j = theta_max j / G, j = 1..G; while its minimum is not
// positive, a second copy of the root nearest the minimising lambda_j (lowest
// index on ties) is appended, at most kInteriorRoots times.  Above theta_max
// the product has the sign (-1)^(count), so an even count gets one more copy
// of theta_max, which keeps p positive there (theta_max can lie a percent
// below lambda_max).  theta holds the k ascending harmonic Ritz values and
// receives the copies after them; kout the new count.  The factors are
// multiplied in list order and the minimum is the first in j, one CTA per
// problem.
constexpr int kDefiniteGrid = 8192;
constexpr int kInteriorRoots = SPHYNX_MAX_ADDED_ROOTS - 1;
constexpr int kRootCap = SPHYNX_MAX_POLY_DEGREE + SPHYNX_MAX_ADDED_ROOTS;

__global__ void __launch_bounds__(256)
k_harmonic_definite(double *theta, int k, int *kout, const int *err, int stride) {
  __shared__ double th[kRootCap];
  __shared__ double wmin[8];
  __shared__ int warg[8];
  __shared__ int kk_s, stop;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  theta += static_cast<int64_t>(blockIdx.x) * stride;
  if (err[blockIdx.x]) {
    if (tid == 0) kout[blockIdx.x] = k;
    return;
  }
  for (int i = tid; i < k; i += blockDim.x) th[i] = theta[i];
  if (tid == 0) kk_s = k;
  __syncthreads();
  const double tmax = th[k - 1];
  for (int add = 0; add < kInteriorRoots; ++add) {
    const int kk = kk_s;
    double best = INFINITY;
    int barg = INT_MAX;
    for (int j = tid + 1; j <= kDefiniteGrid; j += blockDim.x) {
      const double lam = (tmax * static_cast<double>(j)) / static_cast<double>(kDefiniteGrid);
      double pi = 1.0;
      for (int i = 0; i < kk; ++i) pi = pi * (1.0 - lam / th[i]);
      const double p = (1.0 - pi) / lam;
      if (p < best) {
        best = p;
        barg = j;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oa = __shfl_down_sync(0xffffffffu, barg, off);
      if (ov < best || (ov == best && oa < barg)) {
        best = ov;
        barg = oa;
      }
    }
    if (lane == 0) {
      wmin[wid] = best;
      warg[wid] = barg;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w)
        if (wmin[w] < best || (wmin[w] == best && warg[w] < barg)) {
          best = wmin[w];
          barg = warg[w];
        }
      stop = best > 0.0 ? 1 : 0;
      if (!stop) {
        const double lam = (tmax * static_cast<double>(barg)) / static_cast<double>(kDefiniteGrid);
        int near = 0;
        for (int i = 1; i < k; ++i)
          if (fabs(th[i] - lam) < fabs(th[near] - lam)) near = i;
        th[kk] = th[near];
        kk_s = kk + 1;
      }
    }
    __syncthreads();
    if (stop) break;
  }
  if (tid == 0 && kk_s % 2 == 0) {
    th[kk_s] = tmax;
    kk_s = kk_s + 1;
  }
  __syncthreads();
  for (int i = k + tid; i < kk_s; i += blockDim.x) theta[i] = th[i];
  if (tid == 0) kout[blockIdx.x] = kk_s;
}

// Modified Leja order of theta[0..k) (k = kin[problem] when kin is given):
// largest |theta| first, then maximise the product of distances to the roots
// already taken (sum of logs; a repeated root scores -inf until the end);
// ties -> lowest index.  The logs of a step are taken in parallel, one thread
// per candidate.  theta may alias inv: it is read into shared memory first.
// roots[k .. kcap) = +inf and inv[k .. kcap] = 0: the product-form steps of
// an infinite root change nothing, so a batch runs the largest count for all.
__global__ void __launch_bounds__(128)
k_harmonic_leja(const double *theta, int k0, const int *kin, int kcap, double *roots, double *inv, float *invf,
                int *err, int stride) {
  __shared__ double th[kRootCap], score[kRootCap];
  __shared__ int used[kRootCap];
  __shared__ int last;
  const int tid = threadIdx.x;
  const int64_t o = static_cast<int64_t>(blockIdx.x) * stride;   // problem blockIdx.x of a batch
  const int k = kin ? kin[blockIdx.x] : k0;
  theta += o;
  roots += o;
  inv += o;
  invf += o;
  err += blockIdx.x;
  if (*err) return;
  if (tid < k) {
    th[tid] = theta[tid];
    score[tid] = 0.0;
    used[tid] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int first = 0;
    for (int i = 1; i < k; ++i)
      if (fabs(th[i]) > fabs(th[first])) first = i;
    used[first] = 1;
    last = first;
    roots[0] = th[first];
  }
  __syncthreads();
  for (int step = 1; step < k; ++step) {
    if (tid < k && !used[tid]) {
      const double dd = fabs(th[tid] - th[last]);
      score[tid] += dd > 0.0 ? log(dd) : -INFINITY;
    }
    __syncthreads();
    if (tid == 0) {
      int best = -1;
      for (int i = 0; i < k; ++i) {
        if (used[i]) continue;
        if (best < 0 || score[i] > score[best]) best = i;
      }
      used[best] = 1;
      last = best;
      roots[step] = th[best];
    }
    __syncthreads();
  }
  if (tid == 0) {
    int bad = 0;
    for (int i = 0; i < k; ++i) {
      if (!(roots[i] > 0.0) || !isfinite(roots[i])) bad = 1;
      inv[i] = 1.0 / roots[i];
      invf[i] = static_cast<float>(inv[i]);
    }
    for (int i = k; i < kcap; ++i) roots[i] = INFINITY;
    for (int i = k; i <= kcap; ++i) {   // the chain reads inv[i + 1] on its last step
      inv[i] = 0.0;
      invf[i] = 0.f;
    }
    *err = bad ? 2 : 0;
  }
}

}  // namespace

void launch_rayleigh_ritz(cudaStream_t st, const double *ga, const double *gb, int M, int ld, int b,
                          double u_work, SolverState *state, double *y64, void *yt, DT dt,
                          const int *active_override, double *theta_out, int *svqb_out, int mixed, int count) {
  if (M > kMaxM || M < 1) fail(SPHYNX_ERR_INVALID_ARG, "Rayleigh-Ritz size %d outside [1, %d]", M, kMaxM);
  if (b < 1 || b > ld) fail(SPHYNX_ERR_INVALID_ARG, "Rayleigh-Ritz nev %d", b);
  if (count < 1) fail(SPHYNX_ERR_INVALID_ARG, "Rayleigh-Ritz count %d", count);
  const size_t sm = sizeof(RRSmem);
  SPX_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
  k_rayleigh_ritz<<<count, kSmallThreads, sm, st>>>(ga, gb, M, ld, b, u_work, state, active_override, y64, yt,
                                                    dt == DT::F32 ? 1 : 0, theta_out, svqb_out, mixed);
  SPX_LAUNCHED();
}

void launch_harmonic_ritz(cudaStream_t st, const double *alpha, const double *beta2, int k, double *roots,
                          double *inv, float *invf, int *err, int *kout) {
  if (k < 1 || k > SPHYNX_MAX_POLY_DEGREE) fail(SPHYNX_ERR_INVALID_ARG, "polynomial degree %d", k);
  const int kcap = k + SPHYNX_MAX_ADDED_ROOTS;
  k_harmonic_eig<<<k, 32, 0, st>>>(alpha, beta2, k, inv, err, 0);
  SPX_LAUNCHED();
  k_harmonic_definite<<<1, 256, 0, st>>>(inv, k, kout, err, 0);
  SPX_LAUNCHED();
  k_harmonic_leja<<<1, 128, 0, st>>>(inv, k, kout, kcap, roots, inv, invf, err, 0);
  SPX_LAUNCHED();
}

void launch_harmonic_ritz_batch(cudaStream_t st, const double *alpha, const double *beta2, int k, int count,
                                int stride, double *roots, double *inv, float *invf, int *err, int *kout) {
  const int kcap = k + SPHYNX_MAX_ADDED_ROOTS;
  if (k < 1 || k > SPHYNX_MAX_POLY_DEGREE || stride < kcap + 1 || count < 1)
    fail(SPHYNX_ERR_INVALID_ARG, "polynomial degree %d, stride %d, count %d", k, stride, count);
  if (count > 65535) fail(SPHYNX_ERR_UNSUPPORTED, "more than 65535 polynomial setups in one launch");
  k_harmonic_eig<<<dim3(k, count), 32, 0, st>>>(alpha, beta2, k, inv, err, stride);
  SPX_LAUNCHED();
  k_harmonic_definite<<<count, 256, 0, st>>>(inv, k, kout, err, stride);
  SPX_LAUNCHED();
  k_harmonic_leja<<<count, 128, 0, st>>>(inv, k, kout, kcap, roots, inv, invf, err, stride);
  SPX_LAUNCHED();
}

}  // namespace sphynx
