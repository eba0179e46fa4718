// mj.cu -- multi-jagged multisection of the spectral coordinates (Sec. 4).
//
// Rule (exact, integer): a section owning parts [lo, lo + k) splits into
// k_L = ceil(k/2) and k_R = floor(k/2) parts along dimension level mod dims.
// Its points are ordered by the composite key (coordinate, vertex id), the
// coordinate compared as an IEEE value (-0 == +0); the left side is the
// shortest prefix p minimising |k cumW(p) - k_L W| (cumW strictly increasing
// because vertex weights are >= 1).
//
// GPU schedule, one level at a time for all sections at once:
//  * sections are contiguous ranges of a permutation array `perm`;
//  * the split element e (the first point with k cumW >= k_L W) is found by
//    a most-significant-digit radix select over the composite key, 8 bits per
//    pass: a histogram kernel adds (weight, count) of every candidate point
//    into 256 bins per section (shared-memory bins when a CTA's chunk lies in
//    one section), then a warp per section scans its bins and fixes one digit;
//  * a decide kernel compares the prefixes ending just before and just after e,
//    and a scatter kernel moves every point to its child range with
//    warp-aggregated atomics.  The resulting sets (hence part ids) are exact
//    and independent of scheduling.
#include "internal.cuh"

#include <cstring>
#include <mutex>

namespace sphynx {

namespace {

constexpr int kMjThreads = 256;
constexpr int kMjChunk = 4096;

struct MjSec {             // per-section select state (device)
  unsigned long long phi, plo, mhi, mlo;
  long long before, beforecnt, ew, ec;
  long long nleft, wleft;
  int incl, pad;
  unsigned curl, curr;
};

__device__ __forceinline__ unsigned long long ordered_key(const void *coords, int dt, int64_t v, int ldc,
                                                          int dim) {
  if (dt == SPHYNX_DT_F64) {
    double x = static_cast<const double *>(coords)[v * ldc + dim];
    unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    if (x == 0.0) u = 0ull;
    return (u >> 63) ? ~u : (u | (1ull << 63));
  }
  float x = static_cast<const float *>(coords)[v * ldc + dim];
  unsigned u = __float_as_uint(x);
  if (x == 0.0f) u = 0u;
  return static_cast<unsigned long long>((u >> 31) ? ~u : (u | 0x80000000u));
}

struct PassInfo {
  int nd_hi, nd_lo;
};

__device__ __forceinline__ int digit_of(unsigned long long hi, unsigned long long lo, int p, PassInfo pi) {
  if (p < pi.nd_hi) return static_cast<int>((hi >> (8 * (pi.nd_hi - 1 - p))) & 0xFFull);
  const int q = p - pi.nd_hi;
  return static_cast<int>((lo >> (8 * (pi.nd_lo - 1 - q))) & 0xFFull);
}

__device__ __forceinline__ int section_of(const long long *start, int S, int64_t pos) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= pos) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_mj_nan(const void *coords, int dt, int64_t n, int ldc, int dims, unsigned *bad) {
  unsigned b = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int d = 0; d < dims; ++d) {
      if (dt == SPHYNX_DT_F64) {
        if (isnan(static_cast<const double *>(coords)[i * ldc + d])) b = 1;
      } else {
        if (isnan(static_cast<const float *>(coords)[i * ldc + d])) b = 1;
      }
    }
  }
  if (b) atomicOr(bad, 1u);
}

__global__ void k_mj_init(int32_t *perm, int64_t n, const int64_t *vw, unsigned long long *wsum, unsigned *bad) {
  unsigned long long s = 0;
  unsigned b = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    perm[i] = static_cast<int32_t>(i);
    const long long w = vw ? vw[i] : 1;
    if (w < 1) b = 1;
    s += static_cast<unsigned long long>(w);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(wsum, s);
  if (b) atomicOr(bad, 2u);
}

__global__ void k_mj_level0(long long *start, long long *end, long long *W, int64_t n, const unsigned long long *wsum) {
  start[0] = 0;
  end[0] = n;
  W[0] = static_cast<long long>(*wsum);
}

// W[g] = total vertex weight of graph g, vertices [gptr[g], gptr[g+1]); one CTA per graph
__global__ void k_mj_graph_weights(const int64_t *vw, const int64_t *gptr, long long *W) {
  __shared__ unsigned long long red[8];
  const int g = blockIdx.x;
  unsigned long long s = 0;
  for (int64_t i = gptr[g] + threadIdx.x; i < gptr[g + 1]; i += blockDim.x) s += static_cast<unsigned long long>(vw[i]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < 8; ++k) t += red[k];
    W[g] = static_cast<long long>(t);
  }
}

__global__ void k_mj_sel_init(MjSec *sec, int S) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  MjSec z{};
  sec[s] = z;
}

__global__ void __launch_bounds__(kMjThreads)
k_mj_hist(const int32_t *perm, int64_t n, const void *coords, int dt, int ldc, int dim, const int64_t *vw,
          const long long *start, int S, const int *split, const MjSec *sec, int p, PassInfo pi,
          unsigned long long *hist) {
  __shared__ unsigned long long sh[256][2];
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kMjChunk;
  if (c0 >= n) return;
  const int64_t c1 = c0 + kMjChunk < n ? c0 + kMjChunk : n;
  const int s0 = section_of(start, S, c0), s1 = section_of(start, S, c1 - 1);
  const bool one = s0 == s1;
  if (one && !split[s0]) return;
  if (one) {
    sh[threadIdx.x][0] = 0;
    sh[threadIdx.x][1] = 0;
    __syncthreads();
  }
  for (int64_t pos = c0 + threadIdx.x; pos < c1; pos += blockDim.x) {
    const int s = one ? s0 : section_of(start, S, pos);
    if (!split[s]) continue;
    const int32_t v = perm[pos];
    const unsigned long long hi = ordered_key(coords, dt, v, ldc, dim);
    const unsigned long long lo = static_cast<unsigned long long>(v);
    const MjSec &q = sec[s];
    if ((hi & q.mhi) != q.phi || (lo & q.mlo) != q.plo) continue;
    const int d = digit_of(hi, lo, p, pi);
    const unsigned long long w = vw ? static_cast<unsigned long long>(vw[v]) : 1ull;
    if (one) {
      atomicAdd(&sh[d][0], w);
      atomicAdd(&sh[d][1], 1ull);
    } else {
      atomicAdd(&hist[(static_cast<int64_t>(s) * 256 + d) * 2], w);
      atomicAdd(&hist[(static_cast<int64_t>(s) * 256 + d) * 2 + 1], 1ull);
    }
  }
  if (one) {
    __syncthreads();
    const unsigned long long w = sh[threadIdx.x][0], c = sh[threadIdx.x][1];
    if (c) {
      atomicAdd(&hist[(static_cast<int64_t>(s0) * 256 + threadIdx.x) * 2], w);
      atomicAdd(&hist[(static_cast<int64_t>(s0) * 256 + threadIdx.x) * 2 + 1], c);
    }
  }
}

// one warp per section: find the bin holding the first point with
// k (before + cum) >= k_L W, fix that digit, clear the bins
__global__ void k_mj_select(unsigned long long *hist, int S, const int *split, const int *ks, const long long *W,
                            MjSec *sec, int p, PassInfo pi) {
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= S || !split[s]) return;
  const long long k = ks[s], kl = (k + 1) / 2;
  const long long T = kl * W[s];
  MjSec &q = sec[s];
  unsigned long long *h = hist + static_cast<int64_t>(s) * 512;
  long long wb[8], cb[8];
  long long lw = 0, lc = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    wb[u] = static_cast<long long>(h[(lane * 8 + u) * 2]);
    cb[u] = static_cast<long long>(h[(lane * 8 + u) * 2 + 1]);
    lw += wb[u];
    lc += cb[u];
  }
  // exclusive scans of lane sums
  long long pw = lw, pc = lc;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long tw = __shfl_up_sync(0xffffffffu, pw, off);
    const long long tc = __shfl_up_sync(0xffffffffu, pc, off);
    if (lane >= off) { pw += tw; pc += tc; }
  }
  pw -= lw;
  pc -= lc;
  const long long before = q.before, beforecnt = q.beforecnt;
  int found = -1;
  long long fw = 0, fc = 0, ew = 0, ec = 0;
  long long cw = before + pw, cc = beforecnt + pc;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (found < 0 && cb[u] > 0 && k * (cw + wb[u]) >= T) {
      found = lane * 8 + u;
      fw = cw;
      fc = cc;
      ew = wb[u];
      ec = cb[u];
    }
    cw += wb[u];
    cc += cb[u];
  }
  const unsigned ball = __ballot_sync(0xffffffffu, found >= 0);
  const int src = ball ? __ffs(ball) - 1 : 0;
  const int dsel = __shfl_sync(0xffffffffu, found, src);
  fw = __shfl_sync(0xffffffffu, fw, src);
  fc = __shfl_sync(0xffffffffu, fc, src);
  ew = __shfl_sync(0xffffffffu, ew, src);
  ec = __shfl_sync(0xffffffffu, ec, src);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    h[(lane * 8 + u) * 2] = 0;
    h[(lane * 8 + u) * 2 + 1] = 0;
  }
  if (lane == 0 && ball) {
    q.before = fw;
    q.beforecnt = fc;
    q.ew = ew;
    q.ec = ec;
    const unsigned long long d = static_cast<unsigned long long>(dsel);
    if (p < pi.nd_hi) {
      const int sh = 8 * (pi.nd_hi - 1 - p);
      q.phi |= d << sh;
      q.mhi |= 0xFFull << sh;
    } else {
      const int sh = 8 * (pi.nd_lo - 1 - (p - pi.nd_hi));
      q.plo |= d << sh;
      q.mlo |= 0xFFull << sh;
    }
  }
}

// choose the prefix ending just before or just after e; build the next level
__global__ void k_mj_decide(int S, const int *split, const int *ks, const int *child, const long long *start,
                            const long long *end, const long long *W, MjSec *sec, long long *nstart,
                            long long *nend, long long *nW) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int cb = child[s];
  if (!split[s]) {
    nstart[cb] = start[s];
    nend[cb] = end[s];
    nW[cb] = W[s];
    return;
  }
  MjSec &q = sec[s];
  const long long k = ks[s], kl = (k + 1) / 2, w = W[s], T = kl * w;
  long long nl = 0, wl = 0;
  int incl = 0;
  if (w > 0) {
    long long flo = k * q.before - T, fhi = k * (q.before + q.ew) - T;
    flo = flo < 0 ? -flo : flo;
    fhi = fhi < 0 ? -fhi : fhi;
    if (flo <= fhi) {
      nl = q.beforecnt;
      wl = q.before;
    } else {
      nl = q.beforecnt + 1;
      wl = q.before + q.ew;
      incl = 1;
    }
  }
  q.nleft = nl;
  q.wleft = wl;
  q.incl = incl;
  q.curl = 0;
  q.curr = 0;
  nstart[cb] = start[s];
  nend[cb] = start[s] + nl;
  nW[cb] = wl;
  nstart[cb + 1] = start[s] + nl;
  nend[cb + 1] = end[s];
  nW[cb + 1] = w - wl;
}

__global__ void __launch_bounds__(kMjThreads)
k_mj_scatter(const int32_t *perm, int32_t *perm2, int64_t n, const void *coords, int dt, int ldc, int dim,
             const long long *start, int S, const int *split, MjSec *sec) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t pos = base + lane;
    const bool valid = pos < n;
    int s = 0;
    int32_t v = 0;
    long long key = -1;  // group key: section * 2 + side, -1 for lanes with nothing to place
    if (valid) {
      s = section_of(start, S, pos);
      v = perm[pos];
      if (!split[s]) {
        perm2[pos] = v;
      } else {
        const MjSec &q = sec[s];
        const unsigned long long hi = ordered_key(coords, dt, v, ldc, dim);
        const unsigned long long lo = static_cast<unsigned long long>(v);
        const bool less = hi < q.phi || (hi == q.phi && lo < q.plo);
        const bool eq = hi == q.phi && lo == q.plo;
        const bool left = less || (q.incl && eq);
        key = static_cast<long long>(s) * 2 + (left ? 0 : 1);
      }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (key >= 0) {
      const int leader = __ffs(grp) - 1;
      const unsigned rank = __popc(grp & ((1u << lane) - 1u));
      unsigned basei = 0;
      const bool left = (key & 1) == 0;
      if (lane == leader) {
        MjSec &q = sec[s];
        basei = atomicAdd(left ? &q.curl : &q.curr, static_cast<unsigned>(__popc(grp)));
      }
      basei = __shfl_sync(grp, basei, leader);
      const long long off = left ? start[s] : start[s] + sec[s].nleft;
      perm2[off + basei + rank] = v;
    }
  }
}

__global__ void k_mj_parts(const int32_t *perm, int64_t n, const long long *start, int S, const int *lo,
                           int32_t *part) {
  for (int64_t pos = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; pos < n;
       pos += static_cast<int64_t>(gridDim.x) * blockDim.x)
    part[perm[pos]] = lo[section_of(start, S, pos)];
}

int mj_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 8 * kSmCount) g = 8 * kSmCount;
  return static_cast<int>(g < 1 ? 1 : g);
}

struct Level {
  std::vector<int> lo, k, split, child;
};

}  // namespace

size_t mj_scratch_bytes(int64_t n, int K, int count) {
  const size_t Ks = static_cast<size_t>(K);
  return static_cast<size_t>(n) * 8 + Ks * 512 * 8 + Ks * sizeof(MjSec) + Ks * 8 * 6 + 64 +
         Ks * 4 * 4 * 64 /* level tables, up to 64 levels */ + 16 * 256 + 4096 +
         (count > 1 ? static_cast<size_t>(count + 1) * 8 + 256 : 0);
}

void run_mj_scratch(cudaStream_t st, DT dt, const void *coords, int ldc, int dims, int64_t n, const int64_t *vw,
                    int K, int32_t *part, Counters *ctr, void *scratch, const int64_t *h_gptr, int count) {
  if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
  if (K > (1 << 20)) fail(SPHYNX_ERR_UNSUPPORTED, "K > 2^20");
  if (n < 0) fail(SPHYNX_ERR_INVALID_ARG, "n < 0");
  if (count < 1 || (count > 1 && (!h_gptr || K % count != 0)))
    fail(SPHYNX_ERR_INVALID_ARG, "multi-jagged over %d graphs needs their offsets and K a multiple of the count",
         count);
  if (n == 0) return;
  const int k_each = K / count;   // parts of every graph; graph g owns parts [g k_each, (g + 1) k_each)
  if (K == 1) {
    SPX_CUDA(cudaMemsetAsync(part, 0, n * sizeof(int32_t), st));
    return;
  }
  if (dims < 1) fail(SPHYNX_ERR_INVALID_ARG, "multi-jagged needs at least one coordinate");
  if (dt != DT::F32 && dt != DT::F64) fail(SPHYNX_ERR_INVALID_ARG, "coordinates must be float or double");
  const int dti = dt == DT::F64 ? SPHYNX_DT_F64 : SPHYNX_DT_F32;

  // host section tree: (lo, k) per level until every section has k == 1
  std::vector<Level> levels;
  {
    Level l0;
    for (int gi = 0; gi < count; ++gi) {   // one first-level section per graph
      l0.lo.push_back(gi * k_each);
      l0.k.push_back(k_each);
    }
    levels.push_back(l0);
    for (;;) {
      Level &cur = levels.back();
      bool any = false;
      Level nx;
      cur.split.assign(cur.k.size(), 0);
      cur.child.assign(cur.k.size(), 0);
      for (size_t s = 0; s < cur.k.size(); ++s) {
        cur.child[s] = static_cast<int>(nx.k.size());
        if (cur.k[s] >= 2) {
          any = true;
          cur.split[s] = 1;
          const int kl = (cur.k[s] + 1) / 2;
          nx.lo.push_back(cur.lo[s]);
          nx.k.push_back(kl);
          nx.lo.push_back(cur.lo[s] + kl);
          nx.k.push_back(cur.k[s] - kl);
        } else {
          nx.lo.push_back(cur.lo[s]);
          nx.k.push_back(cur.k[s]);
        }
      }
      if (!any) break;
      levels.push_back(nx);
    }
  }
  const int nlev = static_cast<int>(levels.size());
  if (nlev > 64) fail(SPHYNX_ERR_UNSUPPORTED, "too many levels");

  // scratch layout
  char *p = static_cast<char *>(scratch);
  auto take = [&](size_t bytes) {
    char *r = p;
    p += (bytes + 255) & ~static_cast<size_t>(255);
    return r;
  };
  int32_t *perm = reinterpret_cast<int32_t *>(take(n * 4));
  int32_t *perm2 = reinterpret_cast<int32_t *>(take(n * 4));
  unsigned long long *hist = reinterpret_cast<unsigned long long *>(take(static_cast<size_t>(K) * 512 * 8));
  MjSec *sec = reinterpret_cast<MjSec *>(take(static_cast<size_t>(K) * sizeof(MjSec)));
  long long *tab[2][3];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) tab[a][b] = reinterpret_cast<long long *>(take(static_cast<size_t>(K) * 8));
  unsigned long long *misc = reinterpret_cast<unsigned long long *>(take(64));
  // all levels' (k, split, child, lo) tables in one upload
  std::vector<int> host_tab;
  std::vector<size_t> off(nlev);
  for (int l = 0; l < nlev; ++l) {
    off[l] = host_tab.size();
    const Level &L = levels[l];
    const size_t S = L.k.size();
    host_tab.insert(host_tab.end(), L.k.begin(), L.k.end());
    if (L.split.size() == S) host_tab.insert(host_tab.end(), L.split.begin(), L.split.end());
    else host_tab.insert(host_tab.end(), S, 0);
    if (L.child.size() == S) host_tab.insert(host_tab.end(), L.child.begin(), L.child.end());
    else host_tab.insert(host_tab.end(), S, 0);
    host_tab.insert(host_tab.end(), L.lo.begin(), L.lo.end());
  }
  int *dtab = reinterpret_cast<int *>(take(host_tab.size() * 4));
  SPX_CUDA(cudaMemcpyAsync(dtab, host_tab.data(), host_tab.size() * 4, cudaMemcpyHostToDevice, st));
  int64_t *dgptr = count > 1 ? reinterpret_cast<int64_t *>(take(static_cast<size_t>(count + 1) * 8)) : nullptr;
  if (dgptr) {
    if (h_gptr[0] != 0 || h_gptr[count] != n) fail(SPHYNX_ERR_INVALID_ARG, "graph offsets must span [0, n)");
    for (int gi = 0; gi < count; ++gi)
      if (h_gptr[gi + 1] < h_gptr[gi]) fail(SPHYNX_ERR_INVALID_ARG, "graph offsets must not decrease");
    SPX_CUDA(cudaMemcpyAsync(dgptr, h_gptr, static_cast<size_t>(count + 1) * 8, cudaMemcpyHostToDevice, st));
  }
  SPX_CUDA(cudaMemsetAsync(hist, 0, static_cast<size_t>(K) * 512 * 8, st));
  SPX_CUDA(cudaMemsetAsync(misc, 0, 64, st));

  const int g = mj_grid(n);
  k_mj_nan<<<g, 256, 0, st>>>(coords, dti, n, ldc, dims, reinterpret_cast<unsigned *>(misc + 1));
  SPX_LAUNCHED();
  k_mj_init<<<g, 256, 0, st>>>(perm, n, vw, misc, reinterpret_cast<unsigned *>(misc + 1));
  SPX_LAUNCHED();
  unsigned bad = 0;
  SPX_CUDA(cudaMemcpyAsync(&bad, misc + 1, sizeof(bad), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  if (bad & 1u) fail(SPHYNX_ERR_INVALID_ARG, "NaN coordinate");
  if (bad & 2u) fail(SPHYNX_ERR_INVALID_ARG, "vertex weight below 1");
  unsigned long long wtot = 0;
  SPX_CUDA(cudaMemcpyAsync(&wtot, misc, sizeof(wtot), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  // k * cumW must fit in int64: K <= 2^20 and W < 2^40
  if (wtot >= (1ull << 40)) fail(SPHYNX_ERR_UNSUPPORTED, "total vertex weight >= 2^40");
  int64_t launches = 5;
  if (count == 1) {
    k_mj_level0<<<1, 1, 0, st>>>(tab[0][0], tab[0][1], tab[0][2], n, misc);
    SPX_LAUNCHED();
  } else {
    // first level: graph gi is section gi, vertices [gptr[gi], gptr[gi + 1])
    std::vector<long long> hs(count), he(count), hw(count);
    for (int gi = 0; gi < count; ++gi) {
      hs[gi] = h_gptr[gi];
      he[gi] = h_gptr[gi + 1];
      hw[gi] = h_gptr[gi + 1] - h_gptr[gi];
    }
    SPX_CUDA(cudaMemcpyAsync(tab[0][0], hs.data(), count * 8, cudaMemcpyHostToDevice, st));
    SPX_CUDA(cudaMemcpyAsync(tab[0][1], he.data(), count * 8, cudaMemcpyHostToDevice, st));
    if (vw) {
      k_mj_graph_weights<<<count, 256, 0, st>>>(vw, dgptr, tab[0][2]);
      SPX_LAUNCHED();
      ++launches;
    } else {
      SPX_CUDA(cudaMemcpyAsync(tab[0][2], hw.data(), count * 8, cudaMemcpyHostToDevice, st));
    }
    SPX_CUDA(cudaStreamSynchronize(st));   // the host vectors above go out of scope
  }

  int idbits = 1;
  while (idbits < 32 && (1ll << idbits) < n) ++idbits;
  PassInfo pi{dt == DT::F64 ? 8 : 4, (idbits + 7) / 8};
  const int passes = pi.nd_hi + pi.nd_lo;
  const unsigned hist_grid = static_cast<unsigned>((n + kMjChunk - 1) / kMjChunk);
  int cur = 0;
  for (int l = 0; l + 1 < nlev; ++l) {
    const int S = static_cast<int>(levels[l].k.size());
    const int *ks = dtab + off[l];
    const int *split = ks + S;
    const int *child = ks + 2 * S;
    const int dim = l % dims;
    long long *start = tab[cur][0], *end = tab[cur][1], *W = tab[cur][2];
    k_mj_sel_init<<<(S + 127) / 128, 128, 0, st>>>(sec, S);
    SPX_LAUNCHED();
    for (int pss = 0; pss < passes; ++pss) {
      k_mj_hist<<<hist_grid, kMjThreads, 0, st>>>(perm, n, coords, dti, ldc, dim, vw, start, S, split, sec, pss, pi,
                                                  hist);
      SPX_LAUNCHED();
      k_mj_select<<<(S + 7) / 8, 256, 0, st>>>(hist, S, split, ks, W, sec, pss, pi);
      SPX_LAUNCHED();
    }
    long long *nstart = tab[cur ^ 1][0], *nend = tab[cur ^ 1][1], *nW = tab[cur ^ 1][2];
    k_mj_decide<<<(S + 127) / 128, 128, 0, st>>>(S, split, ks, child, start, end, W, sec, nstart, nend, nW);
    SPX_LAUNCHED();
    k_mj_scatter<<<g, kMjThreads, 0, st>>>(perm, perm2, n, coords, dti, ldc, dim, start, S, split, sec);
    SPX_LAUNCHED();
    std::swap(perm, perm2);
    cur ^= 1;
    launches += 3 + 2 * passes;
  }
  const int S = static_cast<int>(levels[nlev - 1].k.size());
  const int *lo = dtab + off[nlev - 1] + 3 * S;
  k_mj_parts<<<g, 256, 0, st>>>(perm, n, tab[cur][0], S, lo, part);
  SPX_LAUNCHED();
  launches += 1;
  if (ctr) ctr->launches += launches;
}

void run_mj(cudaStream_t st, DT dt, const void *coords, int ldc, int dims, int64_t n, const int64_t *vw, int K,
            int32_t *part, Counters *ctr) {
  void *scratch = nullptr;
  const size_t bytes = mj_scratch_bytes(n, K, 1);
  SPX_CUDA(cudaMallocAsync(&scratch, bytes, st));
  try {
    run_mj_scratch(st, dt, coords, ldc, dims, n, vw, K, part, ctr, scratch, nullptr, 1);
  } catch (...) {
    cudaFreeAsync(scratch, st);
    throw;
  }
  SPX_CUDA(cudaFreeAsync(scratch, st));
}

}  // namespace sphynx

extern "C" int sphynx_mj(int32_t dtype, const void *coords, int32_t ldc, int32_t dims, int64_t n,
                         const int64_t *vtx_w, int32_t K, int32_t *part_out, void *stream) {
  using namespace sphynx;
  return guarded([&]() -> int {
    if (n > 0 && (!coords || !part_out)) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (ldc < dims) fail(SPHYNX_ERR_INVALID_ARG, "ldc < dims");
    if (dtype != SPHYNX_DT_F32 && dtype != SPHYNX_DT_F64) fail(SPHYNX_ERR_INVALID_ARG, "dtype");
    // sizes are checked before the scratch is sized from them
    if (n < 0) fail(SPHYNX_ERR_INVALID_ARG, "n < 0");
    if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
    if (K > (1 << 20)) fail(SPHYNX_ERR_UNSUPPORTED, "K > 2^20");
    if (n >= (1LL << 31)) fail(SPHYNX_ERR_UNSUPPORTED, "n >= 2^31");
    run_mj(static_cast<cudaStream_t>(stream), static_cast<DT>(dtype), coords, ldc, dims, n, vtx_w, K, part_out,
           nullptr);
    return SPHYNX_OK;
  });
}

// ---- multi-jagged without any device allocation ------------------------------
//
// Some callers cannot let a library call cudaMalloc: a framework whose own
// caching allocator has already reserved the device's memory, or an
// application that budgets all device memory at start-up and allows no
// allocation afterwards.  For them sphynx_mj_noalloc does the same work as
// sphynx_mj with its scratch (permutations, histograms, section tables) in
// this file-scope device array.  Every GPU that loads the library holds the
// array until the process exits.  The call still synchronises its stream
// twice (run_mj_scratch reads a flag and the total vertex weight back).

constexpr size_t kMjStaticBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_mj_static_scratch[kMjStaticBytes];

namespace {

// Device address of the array, per device.  In host code the array's name is
// only a host-side stand-in, so the address comes from cudaGetSymbolAddress,
// called once per device with that device current.
std::mutex g_mj_static_mutex;
void *g_mj_static_ptr[64] = {nullptr};

void *mj_static_scratch() {
  int dev = 0;
  SPX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) sphynx::fail(SPHYNX_ERR_UNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_mj_static_mutex);
  if (!g_mj_static_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mj_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      sphynx::fail(SPHYNX_ERR_CUDA, "cudaGetSymbolAddress of the multi-jagged scratch failed: %s", cudaGetErrorString(e));
    }
    g_mj_static_ptr[dev] = p;
  }
  return g_mj_static_ptr[dev];
}

}  // namespace

extern "C" int sphynx_mj_noalloc(int32_t dtype, const void *coords, int32_t ldc, int32_t dims, int64_t n,
                                 const int64_t *vtx_w, int32_t K, int32_t *part_out, void *stream) {
  using namespace sphynx;
  return guarded([&]() -> int {
    if (n > 0 && (!coords || !part_out)) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (ldc < dims) fail(SPHYNX_ERR_INVALID_ARG, "ldc < dims");
    if (dtype != SPHYNX_DT_F32 && dtype != SPHYNX_DT_F64) fail(SPHYNX_ERR_INVALID_ARG, "dtype");
    if (n < 0) fail(SPHYNX_ERR_INVALID_ARG, "n < 0");
    if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
    if (K > (1 << 20)) fail(SPHYNX_ERR_UNSUPPORTED, "K > 2^20");
    const size_t need = mj_scratch_bytes(n, K, 1);
    if (need > kMjStaticBytes)
      fail(SPHYNX_ERR_UNSUPPORTED,
           "sphynx_mj_noalloc: n = %lld, K = %d need %zu bytes of scratch, more than its fixed %zu "
           "(e.g. n <= 2^20 with K <= 1024 fits); use sphynx_mj",
           static_cast<long long>(n), K, need, kMjStaticBytes);
    void *scratch = mj_static_scratch();
    // run_mj_scratch clears the histograms and counters it relies on and
    // rewrites everything else it reads
    run_mj_scratch(static_cast<cudaStream_t>(stream), static_cast<DT>(dtype), coords, ldc, dims, n, vtx_w, K,
                   part_out, nullptr, scratch, nullptr, 1);
    return SPHYNX_OK;
  });
}
