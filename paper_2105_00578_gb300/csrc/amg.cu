// amg.cu -- aggregation multigrid preconditioner (Sec. 5.3) with the
// parameters of Sec. 6.2.2: plain aggregation, a degree-3 Chebyshev smoother
// whose largest eigenvalue comes from 10 power-iteration steps with
// eigenvalue ratio 7, at most 5 levels, and the same Chebyshev polynomial as
// the coarse solver with 100 power-iteration steps.
//
// The operator is A = L_C.  With plain aggregation and P the 0/1 aggregate
// indicator, P^T L_C P is the combinatorial Laplacian of the aggregate graph
// whose edge weights are the summed fine weights between two aggregates, so
// every coarse level is again a graph handle and reuses the fused Laplacian
// SpMM.  Readings of the parts the paper leaves to MueLu:
//   aggregation  distance-2 maximal independent set by Luby rounds on keys
//                ((h(v) >> 33) + 1) 2^32 + v, h = SplitMix64 output v + 1 from
//                state mix(seed + 7 gamma + level); a vertex adjacent to a root
//                joins it; every other vertex joins the aggregate of its
//                heaviest already-aggregated neighbour (smallest id on ties);
//   hierarchy    levels are added while a level has more than 2000 vertices,
//                there are fewer than 5 levels and aggregation leaves at most
//                90 % of the vertices;
//   Chebyshev    Saad's Chebyshev acceleration (Iterative Methods for Sparse
//                Linear Systems, Alg. 12.1) of D^{-1} A x = D^{-1} b on
//                [lambda_max / 7, lambda_max], lambda_max = min(1.1 rho, 2)
//                with rho the last Rayleigh quotient of the power iteration
//                (start: SplitMix64 from state mix(seed + 9 gamma + level));
//   cycle        symmetric V-cycle: pre-smooth from zero, restrict, recurse,
//                prolong, post-smooth; the coarsest level smooths from zero.
// Everything is deterministic: reductions run in fixed orders, members of an
// aggregate are listed in a fixed traversal order, and coarse rows are built
// by sorting (column, position) keys.
#include "internal.cuh"

#include <algorithm>

#include <cmath>
#include <vector>

namespace sphynx {

struct AmgLevel {
  sphynx_graph *g = nullptr;   // level 0: the caller's handle; coarser levels: owned
  bool owned = false;
  DevBuf rowptr, col, w;       // coarse levels: the CSR their handle adopts (float weights)
  DevBuf w64, deg64;           // coarse levels: the same weights and their row sums in double
  DevBuf dinv, dinvf;          // 1 / deg (0 where deg = 0), double and float
  DevBuf agg;                  // int32 [n]: aggregate of each vertex (empty on the coarsest level)
  DevBuf mem_ptr;              // int64 [nc + 1]: members of each aggregate ...
  DevBuf mem;                  // int32 [n]: ... in traversal order
  DevBuf blk[5];               // V-cycle blocks: b, x, r, d, y (b and x unused on level 0)
  size_t blk_bytes = 0;
  int64_t n = 0, nc = 0;
  double lam_max = 0;
};

struct AmgHierarchy {
  std::vector<AmgLevel> lv;
  int64_t seed = 0;
  ~AmgHierarchy() {
    // the coarse handles adopt their level's CSR: destroy them before the buffers go
    for (auto &l : lv)
      if (l.owned && l.g) sphynx_destroy(l.g);
  }
};

void amg_free(AmgHierarchy *h) { delete h; }

namespace {

constexpr int64_t kCoarseMax = 2000;
constexpr int kMaxLevels = 5;
constexpr int kChebDegree = 3;
constexpr double kChebRatio = 7.0;
constexpr int kPowerIters = 10;
constexpr int kPowerItersCoarse = 100;
constexpr double kBoost = 1.1;
constexpr int kSortCapMax = 8192;          // entries a coarse row sorts in shared memory
constexpr unsigned long long kRootKey = ~0ull;

unsigned grid1(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

// ---- exclusive scan of int64 counts: out[0..n] with out[n] = total --------
constexpr int kScanItems = 1024;

__global__ void __launch_bounds__(256) k_scan_local(const int64_t *in, int64_t *out, int64_t n, int64_t *bsum) {
  __shared__ int64_t ws[8];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanItems;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int64_t v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = base + 4 * t + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int64_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int64_t woff = 0;
  for (int k = 0; k < w; ++k) woff += ws[k];
  int64_t run = woff + inc - s;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = base + 4 * t + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (t == 255) bsum[blockIdx.x] = woff + inc;
}

__global__ void k_scan_blocks(int64_t *bsum, int64_t nb, int64_t *total) {
  // one thread: the block sums are few (n / 1024)
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t s = bsum[b];
    bsum[b] = run;
    run += s;
  }
  *total = run;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *boff, const int64_t *total) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / kScanItems];
  if (i == 0) out[n] = *total;
}

// out has n + 1 entries; returns the total (synchronises the stream)
int64_t scan_excl(cudaStream_t st, const int64_t *in, int64_t *out, int64_t n) {
  const int64_t nb = (n + kScanItems - 1) / kScanItems;
  DevBuf bs;
  bs.alloc(static_cast<size_t>(nb + 2) * sizeof(int64_t));
  int64_t *bsum = bs.as<int64_t>(), *total = bsum + nb + 1;
  if (n > 0) {
    k_scan_local<<<static_cast<unsigned>(nb), 256, 0, st>>>(in, out, n, bsum);
    SPX_LAUNCHED();
  }
  k_scan_blocks<<<1, 32, 0, st>>>(bsum, nb, total);
  SPX_LAUNCHED();
  k_scan_add<<<grid1(n > 0 ? n : 1), 256, 0, st>>>(out, n, bsum, total);
  SPX_LAUNCHED();
  int64_t h = 0;
  SPX_CUDA(cudaMemcpyAsync(&h, total, sizeof(h), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  return h;
}

// ---- aggregation --------------------------------------------------------------
__global__ void k_keys(int64_t n, uint64_t state, unsigned long long *key) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint64_t h = mix64(state + static_cast<uint64_t>(v + 1) * kGamma);
  key[v] = (((h >> 33) + 1ull) << 32) | static_cast<uint64_t>(v);
}

__device__ __forceinline__ unsigned long long key_of(const unsigned long long *key, const uint8_t *st, int64_t u) {
  const uint8_t s = st[u];
  return s == 1 ? kRootKey : (s == 0 ? key[u] : 0ull);
}

// m1(v) = max over v and its neighbours of k(u)
__global__ void k_mis_m1(int64_t n, const int64_t *rp, const int32_t *col, const unsigned long long *key,
                         const uint8_t *st, unsigned long long *m1) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n) return;
  unsigned long long m = key_of(key, st, v);
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
    const unsigned long long k = key_of(key, st, col[e]);
    m = k > m ? k : m;
  }
  m1[v] = m;
}

// m2(v) = max over v and its neighbours of m1; then the undecided v is ruled
// out (a root within distance 2) or becomes a root (its key is the maximum)
__global__ void k_mis_m2(int64_t n, const int64_t *rp, const int32_t *col, const unsigned long long *key,
                         const unsigned long long *m1, uint8_t *st, unsigned long long *undecided) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  bool still = false;
  if (v < n && st[v] == 0) {
    unsigned long long m = m1[v];
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      const unsigned long long k = m1[col[e]];
      m = k > m ? k : m;
    }
    if (m == kRootKey) st[v] = 2;
    else if (m == key[v]) st[v] = 1;
    else still = true;
  }
  const unsigned b = __ballot_sync(0xffffffffu, still);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(undecided, static_cast<unsigned long long>(__popc(b)));
}

__global__ void k_root_flags(int64_t n, const uint8_t *st, int64_t *flag) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v < n) flag[v] = st[v] == 1 ? 1 : 0;
}

// phase 1: a root takes its own id, a vertex adjacent to a root the root's id
__global__ void k_phase1(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *st, const int64_t *rid,
                         int32_t *a1, int32_t *roots) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (st[v] == 1) {
    a1[v] = static_cast<int32_t>(rid[v]);
    roots[rid[v]] = static_cast<int32_t>(v);
    return;
  }
  int32_t a = -1;
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
    const int32_t u = col[e];
    if (st[u] == 1) {
      a = static_cast<int32_t>(rid[u]);
      break;
    }
  }
  a1[v] = a;
}

// phase 2: the rest join the phase-1 aggregate of the heaviest neighbour,
// the smallest neighbour id on ties; via[v] records that neighbour
__global__ void k_phase2(int64_t n, const int64_t *rp, const int32_t *col, const float *w, const int32_t *a1,
                         int32_t *agg, int32_t *via, int *bad) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (a1[v] >= 0) {
    agg[v] = a1[v];
    via[v] = -1;
    return;
  }
  int32_t best = -1;
  float bw = 0.f;
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
    const int32_t u = col[e];
    if (a1[u] < 0) continue;
    const float we = w ? w[e] : 1.f;
    if (best < 0 || we > bw || (we == bw && u < best)) {
      best = u;
      bw = we;
    }
  }
  if (best < 0) {
    atomicExch(bad, 1);
    agg[v] = 0;
    via[v] = -1;
    return;
  }
  agg[v] = a1[best];
  via[v] = best;
}

// Members of aggregate I in traversal order: the root r, r's neighbours in
// CSR order, then for each of those neighbours u (in the same order) the
// vertices that joined through u, in u's CSR order.
template <bool FILL>
__global__ void k_members(int64_t nc, const int32_t *roots, const int64_t *rp, const int32_t *col,
                          const int32_t *via, int64_t *cnt, const int64_t *mptr, int32_t *mem) {
  const int64_t I = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const int32_t r = roots[I];
  int64_t k = FILL ? mptr[I] : 0;
  if (FILL) mem[k] = r;
  ++k;
  for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
    if (FILL) mem[k] = col[e];
    ++k;
  }
  for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
    const int32_t u = col[e];
    for (int64_t f = rp[u]; f < rp[u + 1]; ++f) {
      const int32_t v = col[f];
      if (via[v] == u) {
        if (FILL) mem[k] = v;
        ++k;
      }
    }
  }
  if (!FILL) cnt[I] = k;
}

// entries (fine edges) a coarse row collects: sum of its members' degrees
__global__ void k_member_entries(int64_t nc, const int64_t *mptr, const int32_t *mem, const int64_t *rp,
                                 int64_t *ent) {
  const int64_t I = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int64_t s = 0;
  for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) s += rp[mem[k] + 1] - rp[mem[k]];
  ent[I] = s;
}

// One coarse row per block: collect (J, position) keys of the members' edges
// to other aggregates, bitonic-sort them in shared memory, and add the
// weights of each J in position order.  The row goes to tmp at an atomic
// cursor with its start and length recorded; a copy kernel places it.
// Rows whose keys fit kSortCapMax entries sort in shared memory; the few
// larger ones (hub aggregates of irregular graphs) sort in a global scratch
// slice of `cap` entries per block (gkey != NULL).  `list` names the
// aggregate of each block.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_coarse_row(const int32_t *list, const int64_t *mptr, const int32_t *mem,
                                                        const int64_t *rp, const int32_t *col, const float *w,
                                                        const double *w64, const int32_t *agg, int64_t cap,
                                                        int64_t *row_cnt, int64_t *row_start,
                                                        unsigned long long *cursor, int32_t *tcol, float *tw,
                                                        double *tw64, unsigned long long *gkey, double *gw) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *key = gkey ? gkey + static_cast<int64_t>(blockIdx.x) * cap
                                 : reinterpret_cast<unsigned long long *>(smem);
  double *wv = gkey ? gw + static_cast<int64_t>(blockIdx.x) * cap : reinterpret_cast<double *>(key + cap);
  __shared__ int64_t s_cnt[THREADS];
  __shared__ int64_t s_base;
  const int t = threadIdx.x;
  const int64_t I = list[blockIdx.x];
  int64_t base = 0;
  for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) {
    const int32_t i = mem[k];
    const int64_t rb = rp[i], re = rp[i + 1];
    for (int64_t e = rb + t; e < re; e += blockDim.x) {
      const int64_t pos = base + (e - rb);
      const int32_t J = agg[col[e]];
      key[pos] = J != static_cast<int32_t>(I) ? ((static_cast<unsigned long long>(J) << 32) | static_cast<uint32_t>(pos))
                                               : kRootKey;
      wv[pos] = w64 ? w64[e] : (w ? static_cast<double>(w[e]) : 1.0);
    }
    base += re - rb;
  }
  for (int64_t p = base + t; p < cap; p += blockDim.x) key[p] = kRootKey;
  __syncthreads();
  for (int64_t kk = 2; kk <= cap; kk <<= 1) {
    for (int64_t j = kk >> 1; j > 0; j >>= 1) {
      for (int64_t i = t; i < cap; i += blockDim.x) {
        const int64_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], b = key[ixj];
          const bool up = (i & kk) == 0;
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // heads of runs of equal J among the valid keys; thread t owns a contiguous chunk
  const int64_t chunk = (cap + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * chunk, hi = lo + chunk < cap ? lo + chunk : cap;
  int64_t nh = 0;
  for (int64_t i = lo; i < hi; ++i) {
    if (key[i] == kRootKey) break;
    if (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32)) ++nh;
  }
  s_cnt[t] = nh;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < THREADS; ++k) {
      const int64_t c = s_cnt[k];
      s_cnt[k] = run;
      run += c;
    }
    s_base = static_cast<int64_t>(atomicAdd(cursor, static_cast<unsigned long long>(run)));
    row_cnt[I] = run;
    row_start[I] = s_base;
  }
  __syncthreads();
  int64_t o = s_base + s_cnt[t];
  for (int64_t i = lo; i < hi; ++i) {
    if (key[i] == kRootKey) break;
    if (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32)) {
      const unsigned long long J = key[i] >> 32;
      double s = 0.0;
      for (int64_t q = i; q < cap && key[q] != kRootKey && (key[q] >> 32) == J; ++q)
        s += wv[static_cast<uint32_t>(key[q] & 0xffffffffull)];
      tcol[o] = static_cast<int32_t>(J);
      tw[o] = static_cast<float>(s);
      tw64[o] = s;
      ++o;
    }
  }
}

// one coarse row per block (64 threads): columns, float and double weights,
// and the double row sum (thread k adds entries k, k + 64, ...; thread 0 adds
// those partial sums in order)
__global__ void k_coarse_place(int64_t nc, const int64_t *row_cnt, const int64_t *row_start, const int64_t *crp,
                               const int32_t *tcol, const float *tw, const double *tw64, int32_t *ccol, float *cw,
                               double *cw64, double *cdeg64) {
  __shared__ double part[64];
  const int64_t I = blockIdx.x;
  if (I >= nc) return;
  const int64_t c = row_cnt[I], s = row_start[I], d = crp[I];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < c; k += blockDim.x) {
    ccol[d + k] = tcol[s + k];
    cw[d + k] = tw[s + k];
    cw64[d + k] = tw64[s + k];
    acc += tw64[s + k];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 64; ++k) t += part[k];
    cdeg64[I] = t;
  }
}

// y = D x - W x with double weights and degrees (a coarse level in FP64), ld columns
__global__ void k_level_spmm64(int64_t n, int ld, const int64_t *rp, const int32_t *col, const double *w,
                               const double *deg, const double *x, double *y, const int *done) {
  if (done && *done) return;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * ld) return;
  const int64_t i = e / ld;
  const int c = static_cast<int>(e - i * ld);
  double acc = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) acc += w[k] * x[static_cast<int64_t>(col[k]) * ld + c];
  y[e] = deg[i] * x[e] - acc;
}

// 1 / deg, 0 where deg = 0
__global__ void k_dinv(int64_t n, const double *deg, double *dinv, float *dinvf) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = deg[i];
  const double v = d > 0.0 ? 1.0 / d : 0.0;
  dinv[i] = v;
  dinvf[i] = static_cast<float>(v);
}

// ---- power iteration on D^{-1} L_C (FP64, fixed-order reductions) -----------
constexpr int kRedGrid = 256;

__global__ void k_rand_pm1(int64_t n, uint64_t state, double *v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t z = mix64(state + static_cast<uint64_t>(i + 1) * kGamma);
  v[i] = 2.0 * (static_cast<double>(z >> 11) * 0x1.0p-53) - 1.0;
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) s += sh[k];
  return s;
}

// mode 0: part = (sum deg v^2, 0); mode 1: part = (sum v y, sum y^2 / deg)
__global__ void __launch_bounds__(256) k_pw_partials(int64_t n, int mode, const double *v, const double *y,
                                                     const double *deg, const double *dinv, double *part) {
  __shared__ double sh[8];
  double a = 0.0, b = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (mode == 0) {
      a += deg[i] * v[i] * v[i];
    } else {
      a += v[i] * y[i];
      b += y[i] * y[i] * dinv[i];
    }
  }
  const double sa = block_sum(a, sh);
  const double sb = block_sum(b, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

// scal[0] = lambda (mode 1), scal[1] = 1 / sqrt(norm^2) (0 for a zero vector)
__global__ void k_pw_final(const double *part, int nb, int mode, double *scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nb; ++k) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  const double nrm2 = mode == 0 ? a : b;
  if (mode == 1) scal[0] = a;
  scal[1] = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
}

// v = s * v (mode 0) or v = s * y / deg (mode 1), s = scal[1]
__global__ void k_pw_next(int64_t n, int mode, const double *y, const double *dinv, const double *scal, double *v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = scal[1];
  v[i] = mode == 0 ? v[i] * s : y[i] * dinv[i] * s;
}

// ---- Chebyshev and the cycle's transfer kernels ----------------------------------
// r = dinv (b - y) (y NULL: dinv b); d = r / theta; x = d (x_zero) or x + d
template <typename T>
__global__ void k_cheb_start(int64_t n, int ld, const T *b, const T *y, const T *dinv, T inv_theta, T *r, T *d,
                             T *x, int x_zero, const int *done) {
  if (done && *done) return;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * ld) return;
  const T di = dinv[e / ld];
  const T rv = di * (y ? b[e] - y[e] : b[e]);
  const T dv = rv * inv_theta;
  r[e] = rv;
  d[e] = dv;
  x[e] = x_zero ? dv : x[e] + dv;
}

// r -= dinv y; d = c1 d + c2 r; x += d
template <typename T>
__global__ void k_cheb_step(int64_t n, int ld, const T *y, const T *dinv, T c1, T c2, T *r, T *d, T *x,
                            const int *done) {
  if (done && *done) return;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * ld) return;
  const T rv = r[e] - dinv[e / ld] * y[e];
  const T dv = c1 * d[e] + c2 * rv;
  r[e] = rv;
  d[e] = dv;
  x[e] += dv;
}

// bc[I] = sum over members i of I, in member order, of b[i] - y[i]
template <typename T>
__global__ void k_restrict(int64_t nc, int ld, const int64_t *mptr, const int32_t *mem, const T *b, const T *y,
                           T *bc, const int *done) {
  if (done && *done) return;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nc * ld) return;
  const int64_t I = e / ld;
  const int c = static_cast<int>(e - I * ld);
  T s = T(0);
  for (int64_t k = mptr[I]; k < mptr[I + 1]; ++k) {
    const int64_t i = mem[k];
    s += b[i * ld + c] - y[i * ld + c];
  }
  bc[e] = s;
}

// x[i] += xc[agg[i]]
template <typename T>
__global__ void k_prolong(int64_t n, int ld, const int32_t *agg, const T *xc, T *x, const int *done) {
  if (done && *done) return;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * ld) return;
  const int64_t i = e / ld;
  x[e] += xc[static_cast<int64_t>(agg[i]) * ld + (e - i * ld)];
}

void level_spmm(sphynx_graph *g, DT dt, const void *x, void *y, int ld, const int *done) {
  SpmmArgs a{};
  a.lap = SPHYNX_COMBINATORIAL;
  a.tin = dt;
  a.ld_x = ld;
  a.ld_y = ld;
  a.bp = ld;
  a.b_true = ld;
  a.x = x;
  a.y = y;
  a.mode = 0;
  a.done = done;
  spmm(g, a);
}

// y = L_C x on one level: FP64 products of a coarse level use its double
// weights and degrees (its handle holds them rounded to float); everything
// else goes through the level's handle and the fused SpMM
void level_product(AmgLevel &L, DT dt, const void *x, void *y, int ld, const int *done) {
  if (dt == DT::F64 && L.w64.p) {
    const int64_t ne = L.n * ld;
    k_level_spmm64<<<grid1(ne), 256, 0, L.g->stream>>>(L.n, ld, L.rowptr.as<int64_t>(), L.col.as<int32_t>(),
                                                        L.w64.as<double>(), L.deg64.as<double>(),
                                                        static_cast<const double *>(x), static_cast<double *>(y),
                                                        done);
    SPX_LAUNCHED();
    L.g->ctr.launches++;
    return;
  }
  level_spmm(L.g, dt, x, y, ld, done);
}

// largest eigenvalue bound of D^{-1} L_C on one level
double power_lambda(AmgLevel &L, int iters, uint64_t state) {
  sphynx_graph *g = L.g;
  cudaStream_t st = g->stream;
  const int64_t n = L.n;
  DevBuf vb, yb, pb;
  vb.alloc(static_cast<size_t>(n) * sizeof(double));
  yb.alloc(static_cast<size_t>(n) * sizeof(double));
  pb.alloc((2 * kRedGrid + 4) * sizeof(double));
  double *v = vb.as<double>(), *y = yb.as<double>(), *part = pb.as<double>(), *scal = part + 2 * kRedGrid;
  const double *deg = L.deg64.p ? L.deg64.as<double>() : g->deg.as<double>(), *dinv = L.dinv.as<double>();
  k_rand_pm1<<<grid1(n), 256, 0, st>>>(n, state, v);
  SPX_LAUNCHED();
  k_pw_partials<<<kRedGrid, 256, 0, st>>>(n, 0, v, nullptr, deg, dinv, part);
  SPX_LAUNCHED();
  k_pw_final<<<1, 32, 0, st>>>(part, kRedGrid, 0, scal);
  SPX_LAUNCHED();
  k_pw_next<<<grid1(n), 256, 0, st>>>(n, 0, nullptr, dinv, scal, v);
  SPX_LAUNCHED();
  SPX_CUDA(cudaMemsetAsync(scal, 0, 2 * sizeof(double), st));
  for (int it = 0; it < iters; ++it) {
    level_product(L, DT::F64, v, y, 1, nullptr);
    k_pw_partials<<<kRedGrid, 256, 0, st>>>(n, 1, v, y, deg, dinv, part);
    SPX_LAUNCHED();
    k_pw_final<<<1, 32, 0, st>>>(part, kRedGrid, 1, scal);
    SPX_LAUNCHED();
    k_pw_next<<<grid1(n), 256, 0, st>>>(n, 1, y, dinv, scal, v);
    SPX_LAUNCHED();
  }
  double lam = 0.0;
  SPX_CUDA(cudaMemcpyAsync(&lam, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  const double b = kBoost * lam;
  return b < 2.0 ? b : 2.0;
}

// aggregate level L; returns the number of aggregates (fills agg, mem_ptr, mem)
int64_t aggregate_level(AmgLevel &L, int level, int64_t seed) {
  sphynx_graph *g = L.g;
  cudaStream_t st = g->stream;
  const int64_t n = L.n;
  DevBuf keyb, m1b, stb, cntb, flagb, ridb, a1b, viab, rootsb;
  keyb.alloc(n * sizeof(unsigned long long));
  m1b.alloc(n * sizeof(unsigned long long));
  stb.alloc(n);
  cntb.alloc(sizeof(unsigned long long) + sizeof(int));
  unsigned long long *key = keyb.as<unsigned long long>(), *m1 = m1b.as<unsigned long long>();
  uint8_t *stt = stb.as<uint8_t>();
  unsigned long long *und = cntb.as<unsigned long long>();
  SPX_CUDA(cudaMemsetAsync(stt, 0, n, st));
  k_keys<<<grid1(n), 256, 0, st>>>(n, mix64(static_cast<uint64_t>(seed) + 7 * kGamma + static_cast<uint64_t>(level)),
                                   key);
  SPX_LAUNCHED();
  // Luby rounds: each round decides at least the undecided vertex of largest key
  for (int64_t round = 0;; ++round) {
    if (round > n + 1) fail(SPHYNX_ERR_CUDA, "multigrid aggregation did not terminate");
    SPX_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), st));
    k_mis_m1<<<grid1(n), 256, 0, st>>>(n, g->rowptr, g->col, key, stt, m1);
    SPX_LAUNCHED();
    k_mis_m2<<<grid1(n), 256, 0, st>>>(n, g->rowptr, g->col, key, m1, stt, und);
    SPX_LAUNCHED();
    unsigned long long h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, und, sizeof(h), cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    if (h == 0) break;
  }
  flagb.alloc(n * sizeof(int64_t));
  ridb.alloc((n + 1) * sizeof(int64_t));
  k_root_flags<<<grid1(n), 256, 0, st>>>(n, stt, flagb.as<int64_t>());
  SPX_LAUNCHED();
  const int64_t nc = scan_excl(st, flagb.as<int64_t>(), ridb.as<int64_t>(), n);
  a1b.alloc(n * sizeof(int32_t));
  rootsb.alloc((nc > 0 ? nc : 1) * sizeof(int32_t));
  k_phase1<<<grid1(n), 256, 0, st>>>(n, g->rowptr, g->col, stt, ridb.as<int64_t>(), a1b.as<int32_t>(),
                                     rootsb.as<int32_t>());
  SPX_LAUNCHED();
  L.agg.alloc(n * sizeof(int32_t));
  viab.alloc(n * sizeof(int32_t));
  int *bad = reinterpret_cast<int *>(und + 1);
  SPX_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_phase2<<<grid1(n), 256, 0, st>>>(n, g->rowptr, g->col, g->w, a1b.as<int32_t>(), L.agg.as<int32_t>(),
                                     viab.as<int32_t>(), bad);
  SPX_LAUNCHED();
  int hbad = 0;
  SPX_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  if (hbad) fail(SPHYNX_ERR_CUDA, "multigrid aggregation left a vertex without an aggregate");
  // members in traversal order
  DevBuf cnt;
  cnt.alloc((nc > 0 ? nc : 1) * sizeof(int64_t));
  L.mem_ptr.alloc((nc + 1) * sizeof(int64_t));
  k_members<false><<<grid1(nc, 128), 128, 0, st>>>(nc, rootsb.as<int32_t>(), g->rowptr, g->col, viab.as<int32_t>(),
                                             cnt.as<int64_t>(), nullptr, nullptr);
  SPX_LAUNCHED();
  const int64_t total = scan_excl(st, cnt.as<int64_t>(), L.mem_ptr.as<int64_t>(), nc);
  if (total != n) fail(SPHYNX_ERR_CUDA, "multigrid aggregates hold %lld of %lld vertices", static_cast<long long>(total),
                       static_cast<long long>(n));
  L.mem.alloc(n * sizeof(int32_t));
  k_members<true><<<grid1(nc, 128), 128, 0, st>>>(nc, rootsb.as<int32_t>(), g->rowptr, g->col, viab.as<int32_t>(),
                                            nullptr, L.mem_ptr.as<int64_t>(), L.mem.as<int32_t>());
  SPX_LAUNCHED();
  L.nc = nc;
  return nc;
}

// the aggregate graph of level L as the CSR of level C (adopted by C's handle)
void coarse_level(AmgLevel &L, AmgLevel &C) {
  sphynx_graph *g = L.g;
  cudaStream_t st = g->stream;
  const int64_t nc = L.nc;
  DevBuf ent, entp;
  ent.alloc(nc * sizeof(int64_t));
  entp.alloc((nc + 1) * sizeof(int64_t));
  k_member_entries<<<grid1(nc), 256, 0, st>>>(nc, L.mem_ptr.as<int64_t>(), L.mem.as<int32_t>(), g->rowptr,
                                              ent.as<int64_t>());
  SPX_LAUNCHED();
  std::vector<int64_t> hent(static_cast<size_t>(nc));
  SPX_CUDA(cudaMemcpyAsync(hent.data(), ent.p, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  // aggregates whose keys fit shared memory, and the rest
  std::vector<int32_t> small, large;
  int64_t mx_s = 0, mx_l = 0, sum = 0;
  for (int64_t I = 0; I < nc; ++I) {
    const int64_t e = hent[static_cast<size_t>(I)];
    sum += e;
    if (e <= kSortCapMax) {
      small.push_back(static_cast<int32_t>(I));
      mx_s = e > mx_s ? e : mx_s;
    } else {
      large.push_back(static_cast<int32_t>(I));
      mx_l = e > mx_l ? e : mx_l;
    }
  }
  if (mx_l >= (int64_t{1} << 31))
    fail(SPHYNX_ERR_UNSUPPORTED, "multigrid: an aggregate has %lld incident entries", static_cast<long long>(mx_l));
  DevBuf rc, rs, cur, tcol, tw, tw64, lists;
  rc.alloc(nc * sizeof(int64_t));
  rs.alloc(nc * sizeof(int64_t));
  cur.alloc(sizeof(unsigned long long));
  tcol.alloc((sum > 0 ? sum : 1) * sizeof(int32_t));
  tw.alloc((sum > 0 ? sum : 1) * sizeof(float));
  tw64.alloc((sum > 0 ? sum : 1) * sizeof(double));
  const double *fw64 = L.w64.p ? L.w64.as<double>() : nullptr;   // the fine level's double weights (coarse levels)
  lists.alloc((small.size() + large.size() + 1) * sizeof(int32_t));
  int32_t *lsmall = lists.as<int32_t>(), *llarge = lsmall + small.size();
  if (!small.empty())
    SPX_CUDA(cudaMemcpyAsync(lsmall, small.data(), small.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (!large.empty())
    SPX_CUDA(cudaMemcpyAsync(llarge, large.data(), large.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  SPX_CUDA(cudaMemsetAsync(cur.p, 0, sizeof(unsigned long long), st));
  if (!small.empty()) {
    // one launch per power-of-two size class, so that a row sorts at the
    // capacity of its own class rather than of the largest aggregate
    int64_t cap0 = 64;
    while (cap0 < mx_s) cap0 <<= 1;
    const size_t smax = static_cast<size_t>(cap0) * (sizeof(unsigned long long) + sizeof(double));
    SPX_CUDA(cudaFuncSetAttribute(k_coarse_row<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smax)));
    std::vector<int32_t> order;
    std::vector<std::pair<int64_t, size_t>> classes;   // (cap, count), caps increasing
    order.reserve(small.size());
    for (int64_t cap = 64, lo = 0; lo < mx_s || cap == 64; lo = cap, cap <<= 1) {
      const size_t first = order.size();
      for (int32_t I : small) {
        const int64_t e = hent[static_cast<size_t>(I)];
        if (e <= cap && (cap == 64 || e > lo)) order.push_back(I);
      }
      if (order.size() > first) classes.emplace_back(cap, order.size() - first);
      if (cap >= cap0) break;
    }
    if (order.size() != small.size()) fail(SPHYNX_ERR_CUDA, "multigrid: size classes lost an aggregate");
    SPX_CUDA(cudaMemcpyAsync(lsmall, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    size_t off = 0;
    for (const auto &c : classes) {
      const size_t sm = static_cast<size_t>(c.first) * (sizeof(unsigned long long) + sizeof(double));
      k_coarse_row<128><<<static_cast<unsigned>(c.second), 128, sm, st>>>(
          lsmall + off, L.mem_ptr.as<int64_t>(), L.mem.as<int32_t>(), g->rowptr, g->col, g->w, fw64,
          L.agg.as<int32_t>(), c.first, rc.as<int64_t>(), rs.as<int64_t>(), cur.as<unsigned long long>(),
          tcol.as<int32_t>(), tw.as<float>(), tw64.as<double>(), nullptr, nullptr);
      SPX_LAUNCHED();
      off += c.second;
    }
    SPX_CUDA(cudaStreamSynchronize(st));   // `order` feeds an asynchronous copy
  }
  if (!large.empty()) {
    // hub aggregates sort in global scratch, grouped by their own power-of-two
    // capacity and launched in chunks whose scratch (12 bytes a key slot) stays
    // within a fixed budget, so that a few huge aggregates cannot size the
    // scratch of all the others
    constexpr size_t kHubBudget = size_t(512) << 20;
    std::vector<std::pair<int64_t, int32_t>> byc;   // (cap, aggregate), caps increasing
    byc.reserve(large.size());
    int64_t capmax = 64;
    for (int32_t I : large) {
      int64_t cap = 64;
      while (cap < hent[static_cast<size_t>(I)]) cap <<= 1;
      byc.emplace_back(cap, I);
      capmax = cap > capmax ? cap : capmax;
    }
    std::sort(byc.begin(), byc.end());
    std::vector<int32_t> order(byc.size());
    for (size_t q = 0; q < byc.size(); ++q) order[q] = byc[q].second;
    SPX_CUDA(cudaMemcpyAsync(llarge, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const size_t slot = sizeof(unsigned long long) + sizeof(double);
    const size_t budget = std::max(kHubBudget, static_cast<size_t>(capmax) * slot);
    DevBuf gk, gwb;
    gk.alloc(budget / slot * sizeof(unsigned long long));
    gwb.alloc(budget / slot * sizeof(double));
    for (size_t q0 = 0; q0 < byc.size();) {
      const int64_t cap = byc[q0].first;
      const size_t per = std::max<size_t>(1, budget / (static_cast<size_t>(cap) * slot));
      size_t q1 = q0;
      while (q1 < byc.size() && byc[q1].first == cap && q1 - q0 < per) ++q1;
      k_coarse_row<1024><<<static_cast<unsigned>(q1 - q0), 1024, 0, st>>>(
          llarge + q0, L.mem_ptr.as<int64_t>(), L.mem.as<int32_t>(), g->rowptr, g->col, g->w, fw64,
          L.agg.as<int32_t>(), cap, rc.as<int64_t>(), rs.as<int64_t>(), cur.as<unsigned long long>(),
          tcol.as<int32_t>(), tw.as<float>(), tw64.as<double>(), gk.as<unsigned long long>(), gwb.as<double>());
      SPX_LAUNCHED();
      q0 = q1;
    }
    SPX_CUDA(cudaStreamSynchronize(st));   // `order` feeds an asynchronous copy; the scratch is freed below
  }
  C.rowptr.alloc((nc + 1) * sizeof(int64_t));
  const int64_t nnz = scan_excl(st, rc.as<int64_t>(), C.rowptr.as<int64_t>(), nc);
  C.col.alloc((nnz > 0 ? nnz : 1) * sizeof(int32_t));
  C.w.alloc((nnz > 0 ? nnz : 1) * sizeof(float));
  C.w64.alloc((nnz > 0 ? nnz : 1) * sizeof(double));
  C.deg64.alloc((nc > 0 ? nc : 1) * sizeof(double));
  k_coarse_place<<<static_cast<unsigned>(nc), 64, 0, st>>>(nc, rc.as<int64_t>(), rs.as<int64_t>(),
                                                           C.rowptr.as<int64_t>(), tcol.as<int32_t>(), tw.as<float>(),
                                                           tw64.as<double>(), C.col.as<int32_t>(), C.w.as<float>(),
                                                           C.w64.as<double>(), C.deg64.as<double>());
  SPX_LAUNCHED();
  sphynx_handle h = nullptr;
  const int code = sphynx_create(C.rowptr.as<int64_t>(), C.col.as<int32_t>(), C.w.as<float>(), nullptr, nc, nnz,
                                 SPHYNX_DEVICE_PTRS, st, &h);
  if (code != SPHYNX_OK) fail(code, "multigrid level %lld: %s", static_cast<long long>(nc), sphynx_last_error());
  C.g = h;
  C.owned = true;
  C.n = nc;
}

void level_dinv(AmgLevel &L) {
  L.dinv.alloc(L.n * sizeof(double));
  L.dinvf.alloc(L.n * sizeof(float));
  const double *deg = L.deg64.p ? L.deg64.as<double>() : L.g->deg.as<double>();
  k_dinv<<<grid1(L.n), 256, 0, L.g->stream>>>(L.n, deg, L.dinv.as<double>(), L.dinvf.as<float>());
  SPX_LAUNCHED();
}

struct ChebCoef {
  double inv_theta;
  double c1[kChebDegree], c2[kChebDegree];
};

ChebCoef cheb_coef(double lam_max) {
  ChebCoef c{};
  if (!(lam_max > 0.0)) return c;   // a level without edges: the smoother returns zero
  const double lam_min = lam_max / kChebRatio;
  const double theta = 0.5 * (lam_max + lam_min), delta = 0.5 * (lam_max - lam_min);
  const double sigma = theta / delta;
  c.inv_theta = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 1; k < kChebDegree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c.c1[k] = rn * rho;
    c.c2[k] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

template <typename T>
void cheb_apply(AmgLevel &L, DT dt, int ld, const T *b, T *x, bool x_zero, T *r, T *d, T *y, const int *done) {
  sphynx_graph *g = L.g;
  cudaStream_t st = g->stream;
  const int64_t ne = L.n * ld;
  const ChebCoef c = cheb_coef(L.lam_max);
  const T *dinv = std::is_same<T, double>::value ? reinterpret_cast<const T *>(L.dinv.p)
                                                 : reinterpret_cast<const T *>(L.dinvf.p);
  if (!x_zero) level_product(L, dt, x, y, ld, done);
  k_cheb_start<T><<<grid1(ne), 256, 0, st>>>(L.n, ld, b, x_zero ? nullptr : y, dinv, static_cast<T>(c.inv_theta), r,
                                             d, x, x_zero ? 1 : 0, done);
  SPX_LAUNCHED();
  for (int k = 1; k < kChebDegree; ++k) {
    level_product(L, dt, d, y, ld, done);
    k_cheb_step<T><<<grid1(ne), 256, 0, st>>>(L.n, ld, y, dinv, static_cast<T>(c.c1[k]), static_cast<T>(c.c2[k]), r, d,
                                              x, done);
    SPX_LAUNCHED();
  }
  g->ctr.launches += kChebDegree;
}

template <typename T>
void vcycle(AmgHierarchy &H, size_t ell, DT dt, int ld, const T *b, T *x, const int *done) {
  AmgLevel &L = H.lv[ell];
  T *r = L.blk[2].as<T>(), *d = L.blk[3].as<T>(), *y = L.blk[4].as<T>();
  if (ell + 1 == H.lv.size()) {
    cheb_apply<T>(L, dt, ld, b, x, true, r, d, y, done);
    return;
  }
  AmgLevel &C = H.lv[ell + 1];
  cudaStream_t st = L.g->stream;
  cheb_apply<T>(L, dt, ld, b, x, true, r, d, y, done);                       // pre-smooth
  level_product(L, dt, x, y, ld, done);                                       // y = A x
  T *bc = C.blk[0].as<T>(), *xc = C.blk[1].as<T>();
  k_restrict<T><<<grid1(C.n * ld), 256, 0, st>>>(C.n, ld, L.mem_ptr.as<int64_t>(), L.mem.as<int32_t>(), b, y, bc,
                                                 done);                       // bc = P^T (b - A x)
  SPX_LAUNCHED();
  vcycle<T>(H, ell + 1, dt, ld, bc, xc, done);
  k_prolong<T><<<grid1(L.n * ld), 256, 0, st>>>(L.n, ld, L.agg.as<int32_t>(), xc, x, done);   // x += P xc
  SPX_LAUNCHED();
  cheb_apply<T>(L, dt, ld, b, x, false, r, d, y, done);                      // post-smooth
  L.g->ctr.launches += 2;
}

void ensure_blocks(AmgHierarchy &H, DT dt, int ld) {
  const size_t es = dt_size(dt);
  for (size_t ell = 0; ell < H.lv.size(); ++ell) {
    AmgLevel &L = H.lv[ell];
    const size_t bytes = static_cast<size_t>(L.n) * ld * es;
    if (L.blk_bytes >= bytes) continue;
    for (int k = (ell == 0 ? 2 : 0); k < 5; ++k) L.blk[k].alloc(bytes);
    L.blk_bytes = bytes;
  }
}

}  // namespace

// Build the hierarchy of g for this seed (rebuild = false: keep one built
// for the same seed).
void amg_setup(sphynx_graph *g, int64_t seed, bool rebuild) {
  if (g->batch.count > 0) fail(SPHYNX_ERR_UNSUPPORTED, "the multigrid preconditioner takes single graphs");
  if (!rebuild && g->amg && g->amg->seed == seed) return;
  if (g->amg) {
    amg_free(g->amg);
    g->amg = nullptr;
  }
  AmgHierarchy *H = new AmgHierarchy();
  try {
    H->seed = seed;
    H->lv.emplace_back();
    H->lv[0].g = g;
    H->lv[0].n = g->n;
    for (int ell = 0;; ++ell) {
      AmgLevel &L = H->lv[ell];
      level_dinv(L);
      bool coarsest = L.n <= kCoarseMax || ell + 1 >= kMaxLevels;
      if (!coarsest) {
        const int64_t nc = aggregate_level(L, ell, seed);
        if (static_cast<double>(nc) > 0.9 * static_cast<double>(L.n)) {
          coarsest = true;
          L.agg.release();
          L.mem_ptr.release();
          L.mem.release();
          L.nc = 0;
        }
      }
      L.lam_max = power_lambda(L, coarsest ? kPowerItersCoarse : kPowerIters,
                               mix64(static_cast<uint64_t>(seed) + 9 * kGamma + static_cast<uint64_t>(ell)));
      if (coarsest) break;
      H->lv.emplace_back();
      coarse_level(H->lv[ell], H->lv[ell + 1]);
    }
  } catch (...) {
    amg_free(H);
    throw;
  }
  g->amg = H;
}

// H = M R: one V-cycle on the n x ld block R (dt F32 or F64)
void amg_apply(sphynx_graph *g, DT dt, const void *r, void *h, int ld, const int *done) {
  if (!g->amg) fail(SPHYNX_ERR_INVALID_ARG, "multigrid preconditioner not set up");
  if (dt == DT::BF16) fail(SPHYNX_ERR_INVALID_ARG, "multigrid blocks are float or double");
  AmgHierarchy &H = *g->amg;
  ensure_blocks(H, dt, ld);
  if (dt == DT::F64)
    vcycle<double>(H, 0, dt, ld, static_cast<const double *>(r), static_cast<double *>(h), done);
  else
    vcycle<float>(H, 0, dt, ld, static_cast<const float *>(r), static_cast<float *>(h), done);
}

// sizes of one level and, on request, its aggregates and CSR (device outputs)
void amg_level_info(sphynx_graph *g, int level, sphynx_amg_level_info *info, int32_t *agg_out, int64_t *rowptr_out,
                    int32_t *col_out, float *w_out) {
  if (!g->amg) fail(SPHYNX_ERR_INVALID_ARG, "multigrid preconditioner not set up");
  AmgHierarchy &H = *g->amg;
  if (level < 0 || level >= static_cast<int>(H.lv.size())) fail(SPHYNX_ERR_INVALID_ARG, "level %d", level);
  AmgLevel &L = H.lv[level];
  cudaStream_t st = g->stream;
  if (info) {
    info->levels = static_cast<int32_t>(H.lv.size());
    info->n = L.n;
    info->nnz = L.g->nnz;
    info->n_next = L.nc;
    info->lambda_max = L.lam_max;
  }
  if (agg_out) {
    if (L.nc == 0) fail(SPHYNX_ERR_INVALID_ARG, "the coarsest level has no aggregates");
    SPX_CUDA(cudaMemcpyAsync(agg_out, L.agg.p, L.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  }
  if (rowptr_out) SPX_CUDA(cudaMemcpyAsync(rowptr_out, L.g->rowptr, (L.n + 1) * sizeof(int64_t),
                                           cudaMemcpyDeviceToDevice, st));
  if (col_out && L.g->nnz)
    SPX_CUDA(cudaMemcpyAsync(col_out, L.g->col, L.g->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (w_out && L.g->nnz) {
    if (!L.g->w) fail(SPHYNX_ERR_INVALID_ARG, "level %d has unit weights", level);
    SPX_CUDA(cudaMemcpyAsync(w_out, L.g->w, L.g->nnz * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  SPX_CUDA(cudaStreamSynchronize(st));
}

}  // namespace sphynx
