// graph.cu -- graph handles: CSR intake and checks, weighted degrees and
// D^{-1/2} (Sec. 3.2), the SpMM row plan, and the exact partition metrics
// (Eq. 1 cutsize and the imbalance of Sec. 3.1).
#include "internal.cuh"

#include <algorithm>

#include <cmath>
#include <cstdarg>
#include <cstring>
#include <memory>

namespace sphynx {

namespace {
thread_local std::string g_error;
}

void set_error_message(const char *msg) { g_error = msg; }
void clear_error() { g_error.clear(); }
const char *last_error_message() { return g_error.c_str(); }

void fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  throw Error{code};
}

void fail_cuda(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", static_cast<int>(e), cudaGetErrorString(e),
           what, file, line);
  g_error = buf;
  throw Error{e == cudaErrorMemoryAllocation ? SPHYNX_ERR_OOM : SPHYNX_ERR_CUDA};
}

void DevBuf::alloc(size_t nbytes) {
  release();
  if (nbytes == 0) return;
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    fail(SPHYNX_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", nbytes, cudaGetErrorString(e));
  }
  bytes = nbytes;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

namespace {

enum : unsigned {
  kBadRowPtr = 1u,
  kBadCol = 2u,
  kSelfLoop = 4u,
  kUnsorted = 8u,
  kAsym = 16u,
  kBadWeight = 32u,
  kBadVWeight = 64u,
};

struct GraphStatsDev {
  unsigned long long max_deg;
  unsigned long long max_wdeg_bits;   // non-negative double as ordered bits
  unsigned long long isolated;
  unsigned long long total_vw;
  int min_exp, max_exp;
  unsigned flags;
  int pad;
};

// row_ptr monotone and in [0, nnz]; every column index in [0, n)
__global__ void k_check_rowptr(const int64_t *rp, int64_t n, int64_t nnz, GraphStatsDev *gs) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t a = rp[i], b = rp[i + 1];
    if (a < 0 || b < a || b > nnz) atomicOr(&gs->flags, kBadRowPtr);
  }
}

__global__ void k_check_cols(const int32_t *col, int64_t nnz, int64_t n, GraphStatsDev *gs) {
  unsigned bad = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < nnz;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = col[e];
    if (j < 0 || static_cast<int64_t>(j) >= n) bad = kBadCol;
  }
  if (bad) atomicOr(&gs->flags, bad);
}

// sortedness, self-loops and symmetry (binary search for (j, i)); weights
// positive, finite and symmetric.  Only runs after the bounds checks passed.
__global__ void k_validate(const int64_t *rp, const int32_t *col, const float *w, int64_t n,
                           GraphStatsDev *gs) {
  unsigned bad = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t a = rp[i], b = rp[i + 1];
    for (int64_t e = a; e < b; ++e) {
      const int32_t j = col[e];
      if (j == i) bad |= kSelfLoop;
      if (e > a && col[e - 1] >= j) bad |= kUnsorted;
      if (w && !(w[e] > 0.f && isfinite(w[e]))) bad |= kBadWeight;
      int64_t lo = rp[j], hi = rp[j + 1] - 1;
      int64_t found = -1;
      while (lo <= hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int32_t c = col[mid];
        if (c == i) { found = mid; break; }
        if (c < i) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0) bad |= kAsym;
      else if (w && w[found] != w[e]) bad |= kAsym;
    }
  }
  if (bad) atomicOr(&gs->flags, bad);
}

__device__ inline unsigned long long dbits(double v) { return static_cast<unsigned long long>(__double_as_longlong(v)); }

__global__ void k_degrees(const int64_t *rp, const float *w, const int64_t *vw, int64_t n, double *deg,
                          float *degf, double *dinv, float *dinvf, double *jinv, float *jinvf,
                          GraphStatsDev *gs) {
  unsigned long long mdeg = 0, mw = 0, iso = 0, tvw = 0;
  int mine = 1 << 20, maxe = -(1 << 20);
  unsigned bad = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t a = rp[i], b = rp[i + 1];
    double d;
    if (w) {
      d = 0.0;
      for (int64_t e = a; e < b; ++e) {
        d += static_cast<double>(w[e]);
        int ex;
        frexpf(w[e], &ex);
        if (w[e] != 0.f) { mine = min(mine, ex); maxe = max(maxe, ex); }
      }
    } else {
      d = static_cast<double>(b - a);
    }
    deg[i] = d;
    degf[i] = static_cast<float>(d);
    const double s = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    dinv[i] = s;
    dinvf[i] = static_cast<float>(s);
    const double jv = d > 0.0 ? 1.0 / d : 1.0;
    jinv[i] = jv;
    jinvf[i] = static_cast<float>(jv);
    mdeg = max(mdeg, static_cast<unsigned long long>(b - a));
    mw = max(mw, dbits(d));
    iso += (b == a) ? 1 : 0;
    if (vw) {
      if (vw[i] < 1) bad |= kBadVWeight;
      tvw += static_cast<unsigned long long>(vw[i]);
    } else {
      tvw += 1;
    }
  }
  // one global atomic per warp and statistic
  for (int off = 16; off > 0; off >>= 1) {
    mdeg = max(mdeg, __shfl_down_sync(0xffffffffu, mdeg, off));
    mw = max(mw, __shfl_down_sync(0xffffffffu, mw, off));
    iso += __shfl_down_sync(0xffffffffu, iso, off);
    tvw += __shfl_down_sync(0xffffffffu, tvw, off);
    mine = min(mine, __shfl_down_sync(0xffffffffu, mine, off));
    maxe = max(maxe, __shfl_down_sync(0xffffffffu, maxe, off));
    bad |= __shfl_down_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) != 0) return;
  atomicMax(&gs->max_deg, mdeg);
  atomicMax(&gs->max_wdeg_bits, mw);
  if (iso) atomicAdd(&gs->isolated, iso);
  atomicAdd(&gs->total_vw, tvw);
  if (w) {
    atomicMin(&gs->min_exp, mine);
    atomicMax(&gs->max_exp, maxe);
  }
  if (bad) atomicOr(&gs->flags, bad);
}

// ---- Eq. 1 cutsize and part weights ----------------------------------------
constexpr int kEvalRun = 64;   // entries per thread step of the cut
__global__ void __launch_bounds__(256)
k_eval(const int64_t *rp, const int32_t *col, const float *w, const int64_t *vw, int64_t n,
       const int32_t *part, int K, int wscale, unsigned long long *cut2, long long *pw, unsigned *badpart,
       int use_smem) {
  extern __shared__ long long spw[];
  if (use_smem) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) spw[k] = 0;
    __syncthreads();
  }
  unsigned long long acc = 0;
  unsigned bad = 0;
  const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  // part weights: one vertex per thread step
  for (int64_t i = tid; i < n; i += nthreads) {
    const int32_t pi = part[i];
    if (pi < 0 || pi >= K) { bad = 1; continue; }
    const long long wv = vw ? vw[i] : 1;
    if (use_smem) atomicAdd(reinterpret_cast<unsigned long long *>(&spw[pi]), static_cast<unsigned long long>(wv));
    else atomicAdd(reinterpret_cast<unsigned long long *>(&pw[pi]), static_cast<unsigned long long>(wv));
  }
  // cut: runs of kEvalRun consecutive entries per thread step, whatever the
  // row lengths; the run's first row comes from a binary search of row_ptr
  const int64_t nnz = rp[n];
  for (int64_t e0 = tid * kEvalRun; e0 < nnz; e0 += nthreads * kEvalRun) {
    int64_t lo = 0, hi = n - 1;                 // last row with rp[row] <= e0
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (rp[mid] <= e0) lo = mid;
      else hi = mid - 1;
    }
    int64_t row = lo;
    const int64_t e1 = e0 + kEvalRun < nnz ? e0 + kEvalRun : nnz;
    for (int64_t e = e0; e < e1; ++e) {
      while (rp[row + 1] <= e) ++row;
      const int32_t pi = part[row], pj = part[col[e]];
      if (pi != pj && pi >= 0 && pi < K) {
        if (w) acc += static_cast<unsigned long long>(llrint(ldexp(static_cast<double>(w[e]), wscale)));
        else acc += 1;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(cut2, acc);
  if (bad) atomicOr(badpart, 1u);
  if (use_smem) {
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x)
      if (spw[k]) atomicAdd(reinterpret_cast<unsigned long long *>(&pw[k]), static_cast<unsigned long long>(spw[k]));
  }
}

// SELL-32 layout of the short rows: per-row degree (0xFF marks a long row)
// and, per 32-row slice, the largest short degree
// Per slice of 32 rows: the largest short-row degree, the number of
// short-row entries, and whether every such entry lies within 32767 of its row
// (then the slice stores 16-bit offsets).  Blocks are whole warps.
__global__ void k_sell_deg(const int64_t *rp, const int32_t *col, int64_t n, uint8_t *sdeg, int *smax, int *ssum,
                           int *sfit) {
  const int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  int d = 0, sd = 0xFF;
  bool fit = true;
  if (row < n) {
    const int64_t dd = rp[row + 1] - rp[row];
    d = dd > (1 << 30) ? (1 << 30) : static_cast<int>(dd);
    sd = d > kShortDeg ? 0xFF : d;
    sdeg[row] = static_cast<uint8_t>(sd);
    if (sd != 0xFF) {
      const int64_t b = rp[row];
      for (int t = 0; t < d; ++t) {
        const int64_t off = static_cast<int64_t>(col[b + t]) - row;
        fit = fit && off >= -32768 && off <= 32767;
      }
    }
  }
  int m = sd == 0xFF ? 0 : d;
  int s = m;
  for (int off = 16; off > 0; off >>= 1) {
    m = max(m, __shfl_down_sync(0xffffffffu, m, off));
    s += __shfl_down_sync(0xffffffffu, s, off);
  }
  fit = __all_sync(0xffffffffu, fit);
  if ((threadIdx.x & 31) == 0 && row < n) {
    smax[row >> 5] = m;
    ssum[row >> 5] = s;
    sfit[row >> 5] = fit ? 1 : 0;
  }
}

__global__ void k_sell_fill(const int64_t *rp, const int32_t *col, const float *w, int64_t n, const uint8_t *sdeg,
                            const int64_t *sptr, const int64_t *cptr, int16_t *scol, float *sw) {
  const int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (row >= n) return;
  const int d = sdeg[row];
  if (d == 0xFF) return;
  const int64_t slice = row >> 5, lane = row & 31, src = rp[row];
  const int64_t cp = cptr[slice];
  if (cp < 0) {
    int16_t *c16 = scol + (~cp) + lane;
    for (int t = 0; t < d; ++t) c16[32 * t] = static_cast<int16_t>(static_cast<int64_t>(col[src + t]) - row);
  } else {
    int32_t *c32 = reinterpret_cast<int32_t *>(scol + cp) + lane;
    for (int t = 0; t < d; ++t) c32[32 * t] = col[src + t];
  }
  if (w) {
    const int64_t b = sptr[slice] + lane;
    for (int t = 0; t < d; ++t) sw[b + 32 * t] = w[src + t];
  }
}

// Shared-pattern test of one 32-row slice (a warp per slice): the lanes walk
// their rows' sorted short-row offsets col - row in step, and each round takes
// the smallest head among the lanes as the next union value U[k]; a lane whose
// head equals it sets bit k of its mask and advances.  Returns the union size
// (at most 31) or -1 when the union is larger or an offset needs more than 16
// bits.  Long rows and padding lanes take no part (bit 31 of their mask).
__device__ int slice_pattern(const int64_t *rp, const int32_t *col, int64_t n, const uint8_t *sdeg, int64_t slice,
                             int lane, unsigned *mask_out, int *u_out) {
  const int64_t row = slice * 32 + lane;
  const bool short_row = row < n && sdeg[row] != 0xFF;
  const int d = short_row ? sdeg[row] : 0;
  const int64_t rb = short_row ? rp[row] : 0;
  unsigned mk = short_row ? 0u : 0x80000000u;
  int myu = 0, nu = 0, t = 0;
  bool ok = true;
  for (;;) {
    int cand = 0x7fffffff;
    if (t < d) {
      const int64_t off = static_cast<int64_t>(col[rb + t]) - row;
      if (off < -32768 || off > 32767) ok = false;
      cand = static_cast<int>(off);
    }
    if (!__all_sync(0xffffffffu, ok)) return -1;
    const int m = __reduce_min_sync(0xffffffffu, cand);
    if (m == 0x7fffffff) break;
    if (nu == 31) return -1;
    if (lane == nu) myu = m;
    if (cand == m) {
      mk |= 1u << nu;
      ++t;
    }
    ++nu;
  }
  *mask_out = mk;
  *u_out = myu;
  return nu;
}

__global__ void k_sell_pattern(const int64_t *rp, const int32_t *col, int64_t n, const uint8_t *sdeg, int *nu_out) {
  const int64_t slice = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slice * 32 >= n) return;   // uniform per warp
  unsigned mk;
  int u;
  const int nu = slice_pattern(rp, col, n, sdeg, slice, lane, &mk, &u);
  if (lane == 0) nu_out[slice] = nu;
}

// writes the shared-pattern blocks: U (32 int16) then the 32 lane masks
__global__ void k_pat_fill(const int64_t *rp, const int32_t *col, int64_t n, const uint8_t *sdeg,
                           const int64_t *pcptr, int16_t *pcol) {
  const int64_t slice = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slice * 32 >= n) return;   // uniform per warp
  const int64_t cp = pcptr[slice];
  if (cp < kPatternTag) return;
  unsigned mk;
  int u;
  const int nu = slice_pattern(rp, col, n, sdeg, slice, lane, &mk, &u);
  int16_t *blk = pcol + (cp - kPatternTag);
  blk[lane] = static_cast<int16_t>(lane < nu ? u : 0);
  reinterpret_cast<unsigned *>(blk + 32)[lane] = mk;
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 8 * kSmCount) g = 8 * kSmCount;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// Rows with more than kShortDeg neighbours: those with at most med_max go to
// the medium-row units (a group of lanes per row), the rest to long-row work
// items (a warp per 1024-entry item).  med_max = kShortDeg sends them all to
// the items.
void build_plan(sphynx_graph *g, const int64_t *host_rowptr, int med_max) {
  SpmmPlan &p = g->plan;
  p.n_long = 0;
  p.n_items = 0;
  p.n_med = 0;
  p.n_units = 0;
  p.med_bytes = 0;
  p.long_bytes = 0;
  p.med_max = med_max;
  if (g->max_degree <= kShortDeg) return;
  std::vector<int64_t> rp_copy;
  const int64_t *rp = host_rowptr;
  if (!rp) {
    rp_copy.resize(static_cast<size_t>(g->n) + 1);
    SPX_CUDA(cudaMemcpyAsync(rp_copy.data(), g->rowptr, (g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    rp = rp_copy.data();
  }
  // medium rows: sorted by degree (descending, row id on ties); a row of d
  // entries gets G = the smallest power of two with d <= G kGroupPerLane (at
  // most 32) lanes, and the rows of one G fill warp units of 32 / G rows
  std::vector<std::pair<int64_t, int32_t>> med;   // (-degree, row)
  for (int64_t i = 0; i < g->n; ++i) {
    const int64_t dg = rp[i + 1] - rp[i];
    if (dg > kShortDeg && dg <= med_max) med.emplace_back(-dg, static_cast<int32_t>(i));
  }
  std::sort(med.begin(), med.end());
  p.n_med = static_cast<int64_t>(med.size());
  if (p.n_med > 0) {
    std::vector<int32_t> grow(med.size());
    std::vector<int32_t> units;   // pairs {first, log2 G | count << 8}
    double entries = 0;
    auto lg_of = [](int64_t d) {
      int lg = 0;
      while (lg < 5 && (int64_t{kGroupPerLane} << lg) < d) ++lg;
      return lg;
    };
    for (int64_t k = 0; k < p.n_med;) {
      const int lg = lg_of(-med[k].first);
      const int cap = 32 >> lg;
      int cnt = 0;
      const int64_t first = k;
      while (k < p.n_med && cnt < cap && lg_of(-med[k].first) == lg) {
        grow[k] = med[k].second;
        entries += static_cast<double>(-med[k].first);
        ++k;
        ++cnt;
      }
      units.push_back(static_cast<int32_t>(first));
      units.push_back(lg | (cnt << 8));
    }
    p.n_units = static_cast<int64_t>(units.size() / 2);
    p.grp_row.alloc(grow.size() * sizeof(int32_t));
    p.grp_unit.alloc(units.size() * sizeof(int32_t));
    SPX_CUDA(cudaMemcpyAsync(p.grp_row.p, grow.data(), grow.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             g->stream));
    SPX_CUDA(cudaMemcpyAsync(p.grp_unit.p, units.data(), units.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));   // the host vectors go out of scope
    // real entries' indices (and weights), the row ids and row pointers, the units
    p.med_bytes = entries * (g->weighted ? 8.0 : 4.0) + static_cast<double>(p.n_med) * 20.0 +
                  static_cast<double>(p.n_units) * 8.0;
  }
  std::vector<int64_t> items, split;
  int64_t nnz_long = 0;
  for (int64_t i = 0; i < g->n; ++i) {
    const int64_t a = rp[i], b = rp[i + 1];
    if (b - a <= med_max) continue;
    nnz_long += b - a;
    const int64_t first = static_cast<int64_t>(items.size() / 4);
    int64_t cnt = 0;
    for (int64_t s = a; s < b; s += kLongChunk) {
      items.push_back(i);
      items.push_back(s);
      items.push_back(s + kLongChunk < b ? s + kLongChunk : b);
      items.push_back(first + cnt);
      ++cnt;
    }
    split.push_back(i);
    split.push_back(first);
    split.push_back(cnt);
  }
  p.n_items = static_cast<int64_t>(items.size() / 4);
  p.n_long = static_cast<int64_t>(split.size() / 3);
  p.long_bytes = static_cast<double>(nnz_long) * (g->weighted ? 8.0 : 4.0) + 32.0 * static_cast<double>(p.n_items) +
                 24.0 * static_cast<double>(p.n_long);
  if (p.n_items > 0) {
    p.items.alloc(items.size() * sizeof(int64_t));
    p.split.alloc(split.size() * sizeof(int64_t));
    SPX_CUDA(cudaMemcpyAsync(p.items.p, items.data(), items.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                             g->stream));
    SPX_CUDA(cudaMemcpyAsync(p.split.p, split.data(), split.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                             g->stream));
    p.partials.alloc(static_cast<size_t>(p.n_items) * 16 * sizeof(double));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
  }
}

void build_sell(sphynx_graph *g) {
  SpmmPlan &p = g->plan;
  const int64_t n = g->n, slices = (n + 31) / 32;
  p.sell_deg.alloc(static_cast<size_t>(n));
  DevBuf sstat;
  sstat.alloc(static_cast<size_t>(slices) * 3 * sizeof(int));
  int *smax = sstat.as<int>(), *ssum = smax + slices, *sfit = ssum + slices;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  k_sell_deg<<<blocks, 256, 0, g->stream>>>(g->rowptr, g->col, n, p.sell_deg.as<uint8_t>(), smax, ssum, sfit);
  SPX_LAUNCHED();
  std::vector<int> hstat(static_cast<size_t>(slices) * 3);
  SPX_CUDA(cudaMemcpyAsync(hstat.data(), sstat.p, hstat.size() * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  SPX_CUDA(cudaStreamSynchronize(g->stream));
  const int *hmax = hstat.data(), *hsum = hmax + slices, *hfit = hsum + slices;
  std::vector<int64_t> hptr(static_cast<size_t>(slices) + 1, 0), hcptr(static_cast<size_t>(slices), 0);
  int64_t units = 0, narrow = 0;
  double idx_bytes = 0, entries = 0;
  for (int64_t s = 0; s < slices; ++s) {
    hptr[s + 1] = hptr[s] + 32 * static_cast<int64_t>(hmax[s]);
    if (hfit[s]) {
      hcptr[s] = ~units;
      units += 32 * static_cast<int64_t>(hmax[s]);
      ++narrow;
      idx_bytes += 2.0 * hsum[s];
    } else {
      units = (units + 63) & ~static_cast<int64_t>(63);   // 128-byte aligned rows of 32 indices
      hcptr[s] = units;
      units += 64 * static_cast<int64_t>(hmax[s]);
      idx_bytes += 4.0 * hsum[s];
    }
    entries += hsum[s];
  }
  p.sell_entries = hptr[slices];
  p.sell_narrow = narrow;
  p.short_entries = entries;
  // indices of the real entries, the degree bytes and one slice offset per slice
  // (plus the weights and their offsets on weighted graphs)
  p.sell_bytes = idx_bytes + static_cast<double>(n) + 8.0 * static_cast<double>(slices) +
                 (g->weighted ? 4.0 * entries + 8.0 * static_cast<double>(slices) : 0.0);
  p.sell_ptr.alloc(hptr.size() * sizeof(int64_t));
  p.sell_cptr.alloc(hcptr.size() * sizeof(int64_t) + 8);
  SPX_CUDA(cudaMemcpyAsync(p.sell_ptr.p, hptr.data(), hptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                           g->stream));
  SPX_CUDA(cudaMemcpyAsync(p.sell_cptr.p, hcptr.data(), hcptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                           g->stream));
  p.sell_col.alloc(static_cast<size_t>(units > 0 ? units : 1) * sizeof(int16_t));
  if (g->weighted) p.sell_w.alloc(static_cast<size_t>(p.sell_entries > 0 ? p.sell_entries : 1) * sizeof(float));
  k_sell_fill<<<blocks, 256, 0, g->stream>>>(g->rowptr, g->col, g->w, n, p.sell_deg.as<uint8_t>(),
                                             p.sell_ptr.as<int64_t>(), p.sell_cptr.as<int64_t>(),
                                             p.sell_col.as<int16_t>(), p.sell_w.as<float>());
  SPX_LAUNCHED();
  // the shared-pattern variant (unweighted graphs with at least one such slice)
  p.pat_slices = 0;
  p.pat_all = false;
  p.pat_cptr.release();
  p.pat_col.release();
  if (!g->weighted && slices > 0) {
    DevBuf nub;
    nub.alloc(static_cast<size_t>(slices) * sizeof(int));
    const unsigned wblocks = static_cast<unsigned>((slices * 32 + 255) / 256);
    k_sell_pattern<<<wblocks, 256, 0, g->stream>>>(g->rowptr, g->col, n, p.sell_deg.as<uint8_t>(), nub.as<int>());
    SPX_LAUNCHED();
    std::vector<int> hnu(static_cast<size_t>(slices));
    SPX_CUDA(cudaMemcpyAsync(hnu.data(), nub.p, hnu.size() * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int64_t> pc(static_cast<size_t>(slices));
    int64_t punits = 0, npat = 0;
    double pbytes = 0;
    for (int64_t s = 0; s < slices; ++s) {
      if (hnu[s] >= 0) {
        pc[s] = kPatternTag | punits;
        punits += 96;   // 64 bytes of offsets, 128 bytes of masks
        pbytes += 192.0;
        ++npat;
      } else {
        pc[s] = hcptr[s];
        const double rows = static_cast<double>(std::min<int64_t>(32, n - 32 * s));
        pbytes += (hcptr[s] < 0 ? 2.0 : 4.0) * hsum[s] + rows;
      }
    }
    if (npat > 0) {
      p.pat_slices = npat;
      p.pat_all = npat == slices;
      p.pat_bytes = pbytes + 8.0 * static_cast<double>(slices);
      p.pat_cptr.alloc(pc.size() * sizeof(int64_t));
      p.pat_col.alloc(static_cast<size_t>(punits) * sizeof(int16_t));
      SPX_CUDA(cudaMemcpyAsync(p.pat_cptr.p, pc.data(), pc.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                               g->stream));
      k_pat_fill<<<wblocks, 256, 0, g->stream>>>(g->rowptr, g->col, n, p.sell_deg.as<uint8_t>(),
                                                 p.pat_cptr.as<int64_t>(), p.pat_col.as<int16_t>());
      SPX_LAUNCHED();
    }
  }
  SPX_CUDA(cudaStreamSynchronize(g->stream));
}

// The short-row schedule is a property of the graph's structure: both are
// timed at create on a float 8-column product and the faster serves every
// later product of the handle.
// The autotuner: at create, times both short-row schedules and, on graphs with
// rows longer than kShortDeg, the medium-row ceilings {kShortDeg, 128, kMedDeg}
// on a float 8-column product, and keeps the fastest combination; when that is
// SELL-32, it then times the slice strides 1 .. 16 and keeps the fastest.
void autotune_spmm(sphynx_graph *g, const int64_t *host_rowptr) {
  const int64_t n = g->n;
  const int ld = 8;
  DevBuf x, y;
  x.alloc(static_cast<size_t>(n) * ld * sizeof(float));
  y.alloc(static_cast<size_t>(n) * ld * sizeof(float));
  SPX_CUDA(cudaMemsetAsync(x.p, 0, static_cast<size_t>(n) * ld * sizeof(float), g->stream));
  SpmmArgs a{};
  a.lap = SPHYNX_COMBINATORIAL;
  a.tin = DT::F32;
  a.ld_x = ld;
  a.ld_y = ld;
  a.bp = ld;
  a.b_true = ld;
  a.x = x.p;
  a.y = y.p;
  std::vector<int> ceilings{kMedDeg};
  if (g->max_degree > kShortDeg) ceilings = {kShortDeg, 128, kMedDeg};
  std::vector<int64_t> rp_copy;
  const int64_t *rp = host_rowptr;
  if (!rp && ceilings.size() > 1) {
    rp_copy.resize(static_cast<size_t>(n) + 1);
    SPX_CUDA(cudaMemcpyAsync(rp_copy.data(), g->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    rp = rp_copy.data();
  }
  float best = 1e30f;
  int best_ceiling = kMedDeg;
  SpmmTuning best_t{};
  g->plan.sell_ls = 0;   // schedules and ceilings are compared in natural slice order
  for (int c : ceilings) {
    if (ceilings.size() > 1) build_plan(g, rp, c);
    const SpmmTuning t = spmm_tune(g, a);
    const float us = t.us[t.variant];
    if (us < best) {
      best = us;
      best_ceiling = c;
      best_t = t;
    }
  }
  if (ceilings.size() > 1 && best_ceiling != ceilings.back()) build_plan(g, rp, best_ceiling);
  g->plan.tuned_variant = best_t.variant;
  for (int v = 0; v < kSpmmVariants; ++v) g->plan.tuned_us[v] = best_t.us[v];
  for (float &u : g->plan.tuned_ls_us) u = 0.f;
  if (best_t.variant != kCsrStaged) spmm_tune_sell_stride(g, a);
  SPX_CUDA(cudaStreamSynchronize(g->stream));
}

}  // namespace

void eval_partition(sphynx_graph *g, const int32_t *part, int K, double *cut, double *cut2, double *imb) {
  if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
  if (g->weighted && !g->wexact)
    fail(SPHYNX_ERR_UNSUPPORTED, "edge weights span too many binary orders for an exact cut");
  const size_t need = 64 + static_cast<size_t>(K) * sizeof(long long);
  char *ws = static_cast<char *>(g->workspace("eval", need, false));
  SPX_CUDA(cudaMemsetAsync(ws, 0, need, g->stream));
  unsigned long long *d_cut = reinterpret_cast<unsigned long long *>(ws);
  unsigned *d_bad = reinterpret_cast<unsigned *>(ws + 8);
  long long *d_pw = reinterpret_cast<long long *>(ws + 64);
  const int use_smem = K <= 4096 ? 1 : 0;
  const size_t sm = use_smem ? K * sizeof(long long) : 0;
  k_eval<<<grid_for(g->n), 256, sm, g->stream>>>(g->rowptr, g->col, g->w, g->vw, g->n, part, K, g->wscale, d_cut,
                                                 d_pw, d_bad, use_smem);
  SPX_LAUNCHED();
  g->ctr.launches++;
  std::vector<char> host(need);
  SPX_CUDA(cudaMemcpyAsync(host.data(), ws, need, cudaMemcpyDeviceToHost, g->stream));
  SPX_CUDA(cudaStreamSynchronize(g->stream));
  unsigned bad;
  memcpy(&bad, host.data() + 8, sizeof(bad));
  if (bad) fail(SPHYNX_ERR_INVALID_ARG, "part ids outside [0, K)");
  unsigned long long c2;
  memcpy(&c2, host.data(), sizeof(c2));
  const long long *pw = reinterpret_cast<const long long *>(host.data() + 64);
  long long mx = 0, tot = 0;
  for (int k = 0; k < K; ++k) {
    mx = pw[k] > mx ? pw[k] : mx;
    tot += pw[k];
  }
  const double twice = ldexp(static_cast<double>(c2), g->weighted ? -g->wscale : 0);
  if (cut2) *cut2 = twice;
  if (cut) *cut = ldexp(static_cast<double>(c2), g->weighted ? -(g->wscale + 1) : -1);
  if (imb) *imb = (static_cast<double>(mx) * static_cast<double>(K)) / static_cast<double>(tot);
}

}  // namespace sphynx

using namespace sphynx;

void *sphynx_graph::workspace(const std::string &name, size_t bytes, bool zero) {
  DevBuf &b = ws[name];
  if (b.bytes < bytes) {
    b.alloc(bytes);
    zero = true;
  }
  if (zero && bytes) SPX_CUDA(cudaMemsetAsync(b.p, 0, bytes, stream));
  return b.p;
}

extern "C" {

const char *sphynx_last_error(void) { return sphynx::last_error_message(); }

void sphynx_default_options(sphynx_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->laplacian = SPHYNX_COMBINATORIAL;
  opt->precond = SPHYNX_PRECOND_JACOBI;
  opt->poly_degree = 25;
  opt->precision = SPHYNX_FP64;
  opt->init = SPHYNX_INIT_RANDOM;
  opt->max_iter = 1000;
  opt->tol = 1e-3;
  opt->seed = 1;
  opt->flags = 0;
  opt->sync_every = 0;
  opt->conv = SPHYNX_CONV_REL_THETA;
}

int sphynx_create(const int64_t *row_ptr, const int32_t *col, const float *edge_w, const int64_t *vtx_w,
                  int64_t n, int64_t nnz, uint32_t flags, void *stream, sphynx_handle *out) {
  return guarded([&]() -> int {
    if (!out) fail(SPHYNX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || nnz < 0) fail(SPHYNX_ERR_INVALID_ARG, "n must be >= 1 and nnz >= 0");
    if (n >= (1LL << 31) - 1) fail(SPHYNX_ERR_UNSUPPORTED, "n >= 2^31 - 1");
    if (nnz >= (1LL << 40)) fail(SPHYNX_ERR_UNSUPPORTED, "nnz >= 2^40");
    if (!row_ptr || (nnz > 0 && !col)) fail(SPHYNX_ERR_INVALID_ARG, "row_ptr/col is NULL");
    const bool dev = (flags & SPHYNX_DEVICE_PTRS) != 0;
    if (!dev && (row_ptr[0] != 0 || row_ptr[n] != nnz))
      fail(SPHYNX_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] = nnz");
    std::unique_ptr<sphynx_graph> g(new sphynx_graph());
    SPX_CUDA(cudaGetDevice(&g->device));
    g->stream = static_cast<cudaStream_t>(stream);
    g->n = n;
    g->nnz = nnz;
    g->weighted = edge_w != nullptr;
    g->has_vw = vtx_w != nullptr;
    if (dev) {
      // the SpMM stages column indices and weights with 16-byte loads
      if (reinterpret_cast<uintptr_t>(col) % 16 || reinterpret_cast<uintptr_t>(edge_w) % 16 ||
          reinterpret_cast<uintptr_t>(row_ptr) % 8 || reinterpret_cast<uintptr_t>(vtx_w) % 8)
        fail(SPHYNX_ERR_INVALID_ARG, "adopted device arrays must be 16-byte (col, weights) / 8-byte aligned");
      g->rowptr = row_ptr;
      g->col = col;
      g->w = edge_w;
      g->vw = vtx_w;
    } else {
      g->own_rowptr.alloc((n + 1) * sizeof(int64_t));
      SPX_CUDA(cudaMemcpyAsync(g->own_rowptr.p, row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
      g->rowptr = g->own_rowptr.as<int64_t>();
      g->own_col.alloc((nnz > 0 ? nnz : 1) * sizeof(int32_t));
      if (nnz) SPX_CUDA(cudaMemcpyAsync(g->own_col.p, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
      g->col = g->own_col.as<int32_t>();
      if (edge_w) {
        g->own_w.alloc((nnz > 0 ? nnz : 1) * sizeof(float));
        if (nnz) SPX_CUDA(cudaMemcpyAsync(g->own_w.p, edge_w, nnz * sizeof(float), cudaMemcpyHostToDevice, g->stream));
        g->w = g->own_w.as<float>();
      }
      if (vtx_w) {
        g->own_vw.alloc(n * sizeof(int64_t));
        SPX_CUDA(cudaMemcpyAsync(g->own_vw.p, vtx_w, n * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
        g->vw = g->own_vw.as<int64_t>();
      }
    }
    g->deg.alloc(n * sizeof(double));
    g->degf.alloc(n * sizeof(float));
    g->dinv.alloc(n * sizeof(double));
    g->dinvf.alloc(n * sizeof(float));
    g->jinv.alloc(n * sizeof(double));
    g->jinvf.alloc(n * sizeof(float));
    SPX_CUDA(cudaMallocHost(&g->host_flag, 256));

    DevBuf gsb;
    gsb.alloc(sizeof(GraphStatsDev));
    GraphStatsDev init{};
    init.min_exp = 1 << 20;
    init.max_exp = -(1 << 20);
    SPX_CUDA(cudaMemcpyAsync(gsb.p, &init, sizeof(init), cudaMemcpyHostToDevice, g->stream));
    GraphStatsDev *gs = gsb.as<GraphStatsDev>();
    GraphStatsDev h{};
    // bounds first: nothing indexes col[] through row_ptr before these pass
    k_check_rowptr<<<grid_for(n), 256, 0, g->stream>>>(g->rowptr, n, nnz, gs);
    SPX_LAUNCHED();
    if (nnz) {
      k_check_cols<<<grid_for(nnz), 256, 0, g->stream>>>(g->col, nnz, n, gs);
      SPX_LAUNCHED();
    }
    SPX_CUDA(cudaMemcpyAsync(&h, gs, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    if (h.flags & kBadRowPtr) fail(SPHYNX_ERR_INVALID_ARG, "row_ptr is not non-decreasing within [0, nnz]");
    if (h.flags & kBadCol) fail(SPHYNX_ERR_INVALID_ARG, "column index outside [0, n)");
    if (flags & SPHYNX_VALIDATE) {
      k_validate<<<grid_for(n), 256, 0, g->stream>>>(g->rowptr, g->col, g->w, n, gs);
      SPX_LAUNCHED();
    }
    k_degrees<<<grid_for(n), 256, 0, g->stream>>>(g->rowptr, g->w, g->vw, n, g->deg.as<double>(), g->degf.as<float>(),
                                                  g->dinv.as<double>(), g->dinvf.as<float>(), g->jinv.as<double>(),
                                                  g->jinvf.as<float>(), gs);
    SPX_LAUNCHED();
    SPX_CUDA(cudaMemcpyAsync(&h, gs, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    SPX_CUDA(cudaStreamSynchronize(g->stream));
    if (h.flags & kSelfLoop) fail(SPHYNX_ERR_INVALID_ARG, "self-loop in the adjacency");
    if (h.flags & kUnsorted) fail(SPHYNX_ERR_INVALID_ARG, "column indices not strictly increasing in a row");
    if (h.flags & kBadWeight) fail(SPHYNX_ERR_INVALID_ARG, "edge weight not positive and finite");
    if (h.flags & kAsym) fail(SPHYNX_ERR_NOT_SYMMETRIC, "adjacency is not symmetric");
    if (h.flags & kBadVWeight) fail(SPHYNX_ERR_INVALID_ARG, "vertex weight below 1");
    g->max_degree = static_cast<int64_t>(h.max_deg);
    memcpy(&g->max_wdeg, &h.max_wdeg_bits, sizeof(double));
    g->isolated = static_cast<int64_t>(h.isolated);
    g->total_vw = static_cast<int64_t>(h.total_vw);
    if (g->total_vw >= (1LL << 40)) fail(SPHYNX_ERR_UNSUPPORTED, "total vertex weight >= 2^40");
    if (g->weighted && nnz) {
      // weight * 2^wscale is an integer for every float weight (24-bit mantissa)
      g->wscale = 24 - h.min_exp;
      const double top = ldexp(1.0, h.max_exp + g->wscale) * static_cast<double>(nnz);
      g->wexact = top < 9.0e18;
    }
    build_plan(g.get(), dev ? nullptr : row_ptr, kMedDeg);
    g->plan.prescale = g->max_degree * g->n > 10 * g->nnz;   // irregular: max degree above 10 x the mean
    build_sell(g.get());
    autotune_spmm(g.get(), dev ? nullptr : row_ptr);
    *out = g.release();
    return SPHYNX_OK;
  });
}

void sphynx_destroy(sphynx_handle g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  if (g->amg) amg_free(g->amg);
  for (auto e : g->ctr.ev_pool) cudaEventDestroy(e);
  if (g->host_flag) cudaFreeHost(g->host_flag);
  delete g;
}

int sphynx_get_info(sphynx_handle g, sphynx_graph_info *info) {
  return guarded([&]() -> int {
    if (!g || !info) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->nnz = g->nnz;
    info->max_degree = g->max_degree;
    info->max_wdegree = g->max_wdeg;
    info->total_vweight = g->total_vw;
    info->long_rows = g->plan.n_med + g->plan.n_long;
    info->weighted = g->weighted ? 1 : 0;
    info->spmm_variant = g->plan.tuned_variant;
    info->tuned_us_csr = g->plan.tuned_us[kCsrStaged];
    info->tuned_us_sell = g->plan.tuned_us[kSell32];
    info->tuned_us_pattern = g->plan.pat_slices > 0 ? g->plan.tuned_us[kSellPattern] : 0.f;
    info->sell_pattern_slices = g->plan.pat_slices;
    info->regular = g->max_degree * g->n <= 10 * g->nnz ? 1 : 0;
    info->spmm_med_max = g->plan.med_max;
    info->sell_stride = 1 << g->plan.sell_ls;
    info->sell_slices = (g->n + 31) / 32;
    info->sell_narrow_slices = g->plan.sell_narrow;
    info->spmm_graph_bytes = (g->plan.tuned_variant == kSell32
                                  ? g->plan.sell_bytes
                                  : g->plan.tuned_variant == kSellPattern
                                        ? g->plan.pat_bytes
                                        : 8.0 * static_cast<double>(g->n + 1) +
                                              g->plan.short_entries * (g->weighted ? 8.0 : 4.0)) +
                             g->plan.med_bytes + g->plan.long_bytes;
    return SPHYNX_OK;
  });
}

int sphynx_default_options_for(sphynx_handle g, int32_t precond, sphynx_options *opt) {
  return guarded([&]() -> int {
    if (!g || !opt) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (precond < SPHYNX_PRECOND_NONE || precond > SPHYNX_PRECOND_AMG) fail(SPHYNX_ERR_INVALID_ARG, "precond");
    sphynx_default_options(opt);
    opt->precond = precond;
    const bool regular = g->max_degree * g->n <= 10 * g->nnz;   // max deg <= 10 x (nnz / n), exactly
    if (regular) {
      opt->laplacian = SPHYNX_COMBINATORIAL;
      opt->tol = precond == SPHYNX_PRECOND_AMG ? 1e-2 : 1e-3;
      opt->init = SPHYNX_INIT_RANDOM;
    } else {
      opt->laplacian = precond == SPHYNX_PRECOND_POLY ? SPHYNX_NORMALIZED : SPHYNX_GENERALIZED;
      opt->tol = 1e-2;
      opt->init = SPHYNX_INIT_PIECEWISE;
    }
    return SPHYNX_OK;
  });
}

int sphynx_set_spmm_med_max(sphynx_handle g, int32_t med_max) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    if (med_max < kShortDeg || med_max > kMedDeg) fail(SPHYNX_ERR_INVALID_ARG, "med_max %d", med_max);
    build_plan(g, nullptr, med_max);
    return SPHYNX_OK;
  });
}

int sphynx_set_spmm_variant(sphynx_handle g, int32_t variant) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    if (variant == -1) {
      g->plan.forced = -1;
      autotune_spmm(g, nullptr);
    } else if (variant == kCsrStaged || variant == kSell32 || (variant == kSellPattern && g->plan.pat_slices > 0)) {
      g->plan.forced = variant;
    } else {
      fail(SPHYNX_ERR_INVALID_ARG, "variant %d", variant);
    }
    return SPHYNX_OK;
  });
}

int sphynx_set_spmm_sell_stride(sphynx_handle g, int32_t stride) {
  return guarded([&]() -> int {
    if (!g) fail(SPHYNX_ERR_INVALID_ARG, "NULL handle");
    if (stride == -1) {
      SpmmArgs a{};
      DevBuf x, y;
      const size_t bytes = static_cast<size_t>(g->n) * 8 * sizeof(float);
      x.alloc(bytes);
      y.alloc(bytes);
      SPX_CUDA(cudaMemsetAsync(x.p, 0, bytes, g->stream));
      a.lap = SPHYNX_COMBINATORIAL;
      a.tin = DT::F32;
      a.ld_x = a.ld_y = a.bp = a.b_true = 8;
      a.x = x.p;
      a.y = y.p;
      spmm_tune_sell_stride(g, a);
      SPX_CUDA(cudaStreamSynchronize(g->stream));
      return SPHYNX_OK;
    }
    int ls = 0;
    while (ls < kSellLsCount && (1 << ls) != stride) ++ls;
    if (ls == kSellLsCount) fail(SPHYNX_ERR_INVALID_ARG, "SELL slice stride %d", stride);
    g->plan.sell_ls = ls;
    return SPHYNX_OK;
  });
}

int sphynx_degrees(sphynx_handle g, double *deg_out) {
  return guarded([&]() -> int {
    if (!g || !deg_out) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    SPX_CUDA(cudaMemcpyAsync(deg_out, g->deg.p, g->n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    return SPHYNX_OK;
  });
}

int sphynx_eval(sphynx_handle g, const int32_t *part, int32_t K, double *cut, double *cut_twice,
                double *imbalance) {
  return guarded([&]() -> int {
    if (!g || !part) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (g->batch.orig.p) {   // a reordered batch: the caller's part ids to row order first
      int32_t *rows = static_cast<int32_t *>(g->workspace("eval_rows", static_cast<size_t>(g->n) * 4, false));
      batch_parts_to_rows(g, part, rows);
      eval_partition(g, rows, K, cut, cut_twice, imbalance);
      return SPHYNX_OK;
    }
    eval_partition(g, part, K, cut, cut_twice, imbalance);
    return SPHYNX_OK;
  });
}

}  // extern "C"
