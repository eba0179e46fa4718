// refine.cu -- greedy cut refinement after multi-jagged.
//
// Sec. 7 proposes a greedy improvement step to lower the cut of the spectral
// partition, noting that KL/FM-style refinement is hard to run in parallel on
// a GPU.  This is a parallel, deterministic, balance-constrained greedy step:
//
//   per round, with integer edge weights w * 2^s (the exact cut's fixed point)
//   and integer vertex weights, and cap = floor((1 + eps) W_total / K):
//   1. every vertex of degree <= max_degree finds its best external part b
//      (largest connection, smallest part on ties) and its gain
//      conn(v, b) - conn(v, p[v]); positive gains are candidates;
//   2. a candidate is selected when no candidate neighbour has a higher
//      (gain, -id): the selected vertices are pairwise non-adjacent, so each
//      gain is exactly the cut its move removes;
//   3. a part takes all the selected vertices aimed at it when they fit cap,
//      otherwise only the one of highest priority, if it fits;
//   4. the accepted vertices move.
// Rounds repeat until none moves or max_rounds is reached.  Every decision is
// an integer comparison, a sum, a max or a min, so the result does not depend
// on the order threads run in.
#include "internal.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace sphynx {

namespace {

__device__ __forceinline__ long long edge_units(const float *w, int wscale, int64_t e) {
  return w ? llrint(ldexp(static_cast<double>(w[e]), wscale)) : 1LL;
}

// gain[v] > 0 with target[v] = b for a candidate, else gain 0 and target -1
__global__ void k_ref_gain(int64_t n, const int64_t *rp, const int32_t *col, const float *w, int wscale,
                           const int32_t *part, int max_degree, long long *gain, int32_t *target) {
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t b0 = rp[v], b1 = rp[v + 1];
    const int a = part[v];
    long long gv = 0;
    int tv = -1;
    if (b1 - b0 <= max_degree) {
      long long internal = 0;
      bool boundary = false;
      for (int64_t e = b0; e < b1; ++e) {
        const int q = part[col[e]];
        if (q == a) internal += edge_units(w, wscale, e);
        else boundary = true;
      }
      if (boundary) {
        long long best_c = 0;
        int best_q = -1;
        for (int64_t e = b0; e < b1; ++e) {
          const int q = part[col[e]];
          if (q == a) continue;
          bool seen = false;
          for (int64_t f = b0; f < e && !seen; ++f) seen = part[col[f]] == q;
          if (seen) continue;
          long long c = 0;
          for (int64_t f = e; f < b1; ++f)
            if (part[col[f]] == q) c += edge_units(w, wscale, f);
          if (c > best_c || (c == best_c && c > 0 && q < best_q)) {
            best_c = c;
            best_q = q;
          }
        }
        if (best_q >= 0 && best_c - internal > 0) {
          gv = best_c - internal;
          tv = best_q;
        }
      }
    }
    gain[v] = gv;
    target[v] = tv;
  }
}

__device__ __forceinline__ bool outranks(long long gu, int64_t u, long long gv, int64_t v) {
  return gu > gv || (gu == gv && u < v);
}

// selected candidates: no candidate neighbour outranks them; per target part,
// the weight aimed at it and the highest gain among them
__global__ void k_ref_select(int64_t n, const int64_t *rp, const int32_t *col, const long long *gain,
                             const int32_t *target, const int64_t *vw, unsigned char *sel,
                             unsigned long long *incoming, long long *best_gain) {
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const long long gv = gain[v];
    bool s = gv > 0;
    for (int64_t e = rp[v]; s && e < rp[v + 1]; ++e) {
      const int64_t u = col[e];
      const long long gu = gain[u];
      if (gu > 0 && outranks(gu, u, gv, v)) s = false;
    }
    sel[v] = s ? 1 : 0;
    if (s) {
      const int b = target[v];
      atomicAdd(&incoming[b], static_cast<unsigned long long>(vw ? vw[v] : 1));
      atomicMax(&best_gain[b], gv);
    }
  }
}

// per target part: the lowest id among its selected vertices of the highest gain
__global__ void k_ref_best_id(int64_t n, const unsigned char *sel, const long long *gain, const int32_t *target,
                              const long long *best_gain, int *best_id) {
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (!sel[v]) continue;
    const int b = target[v];
    if (gain[v] == best_gain[b]) atomicMin(&best_id[b], static_cast<int>(v));
  }
}

// accept and apply the moves of this round; stats[0] moves, stats[1] summed gain
__global__ void k_ref_apply(int64_t n, const unsigned char *sel, const long long *gain, const int32_t *target,
                            const int64_t *vw, const long long *wpart, const unsigned long long *incoming,
                            const int *best_id, long long cap, int32_t *part, long long *wnext,
                            unsigned long long *stats) {
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    if (!sel[v]) continue;
    const int b = target[v];
    const long long wv = vw ? vw[v] : 1;
    const bool all_fit = wpart[b] + static_cast<long long>(incoming[b]) <= cap;
    const bool alone_fits = best_id[b] == static_cast<int>(v) && wpart[b] + wv <= cap;
    if (all_fit || alone_fits) {
      const int a = part[v];
      part[v] = b;
      atomicAdd(reinterpret_cast<unsigned long long *>(&wnext[a]), static_cast<unsigned long long>(-wv));
      atomicAdd(reinterpret_cast<unsigned long long *>(&wnext[b]), static_cast<unsigned long long>(wv));
      atomicAdd(&stats[0], 1ull);
      atomicAdd(&stats[1], static_cast<unsigned long long>(gain[v]));
    }
  }
}

__global__ void k_ref_part_weights(int64_t n, const int32_t *part, const int64_t *vw, int K, long long *wp,
                                   unsigned *bad) {
  for (int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; v < n;
       v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int p = part[v];
    if (p < 0 || p >= K) {
      atomicOr(bad, 1u);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long *>(&wp[p]), static_cast<unsigned long long>(vw ? vw[v] : 1));
  }
}

int ref_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 16 * kSmCount) g = 16 * kSmCount;
  return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace

void refine_partition(sphynx_graph *g, int32_t *part, int K, double eps, int max_rounds, int max_degree,
                      int *moves_out, int *rounds_out) {
  if (K < 1) fail(SPHYNX_ERR_INVALID_ARG, "K must be >= 1");
  if (!(eps >= 0.0) || !std::isfinite(eps)) fail(SPHYNX_ERR_INVALID_ARG, "eps must be finite and >= 0");
  if (max_rounds < 0 || max_degree < 0) fail(SPHYNX_ERR_INVALID_ARG, "max_rounds / max_degree < 0");
  if (g->weighted && !g->wexact)
    fail(SPHYNX_ERR_UNSUPPORTED, "edge weights span too many binary orders for exact integer gains");
  cudaStream_t st = g->stream;
  const int64_t n = g->n;
  const int grid = ref_grid(n);
  long long *gain = static_cast<long long *>(g->workspace("rf_gain", static_cast<size_t>(n) * 8 + 8, false));
  int32_t *target = static_cast<int32_t *>(g->workspace("rf_target", static_cast<size_t>(n) * 4 + 4, false));
  unsigned char *sel = static_cast<unsigned char *>(g->workspace("rf_sel", static_cast<size_t>(n) + 16, false));
  // per part: weight now, weight after the round, incoming weight, best gain, best id; then flags and stats
  const size_t kb = static_cast<size_t>(K) * 8;
  char *small = static_cast<char *>(g->workspace("rf_small", 5 * kb + 64, false));
  long long *wpart = reinterpret_cast<long long *>(small);
  long long *wnext = reinterpret_cast<long long *>(small + kb);
  unsigned long long *incoming = reinterpret_cast<unsigned long long *>(small + 2 * kb);
  long long *best_gain = reinterpret_cast<long long *>(small + 3 * kb);
  int *best_id = reinterpret_cast<int *>(small + 4 * kb);
  unsigned *bad = reinterpret_cast<unsigned *>(small + 5 * kb);
  unsigned long long *stats = reinterpret_cast<unsigned long long *>(small + 5 * kb + 16);
  SPX_CUDA(cudaMemsetAsync(small, 0, 5 * kb + 64, st));
  k_ref_part_weights<<<grid, 256, 0, st>>>(n, part, g->vw, K, wnext, bad);
  SPX_LAUNCHED();
  unsigned hbad = 0;
  SPX_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
  SPX_CUDA(cudaStreamSynchronize(st));
  if (hbad) fail(SPHYNX_ERR_INVALID_ARG, "a part id outside [0, K)");
  // cap = floor((1 + eps) W_total / K) in double, as the reading states
  const double total = static_cast<double>(g->total_vw);
  const long long cap = static_cast<long long>(std::floor((1.0 + eps) * total / static_cast<double>(K)));
  std::vector<int> ids_init(static_cast<size_t>(K), 0x7fffffff);
  int moves = 0, rounds = 0;
  g->ctr.launches += 1;
  for (int r = 0; r < max_rounds; ++r) {
    SPX_CUDA(cudaMemcpyAsync(wpart, wnext, kb, cudaMemcpyDeviceToDevice, st));
    SPX_CUDA(cudaMemsetAsync(incoming, 0, kb, st));
    SPX_CUDA(cudaMemsetAsync(best_gain, 0, kb, st));
    SPX_CUDA(cudaMemcpyAsync(best_id, ids_init.data(), static_cast<size_t>(K) * sizeof(int), cudaMemcpyHostToDevice,
                             st));
    SPX_CUDA(cudaMemsetAsync(stats, 0, 16, st));
    k_ref_gain<<<grid, 256, 0, st>>>(n, g->rowptr, g->col, g->w, g->weighted ? g->wscale : 0, part, max_degree, gain,
                                     target);
    SPX_LAUNCHED();
    k_ref_select<<<grid, 256, 0, st>>>(n, g->rowptr, g->col, gain, target, g->vw, sel, incoming, best_gain);
    SPX_LAUNCHED();
    k_ref_best_id<<<grid, 256, 0, st>>>(n, sel, gain, target, best_gain, best_id);
    SPX_LAUNCHED();
    k_ref_apply<<<grid, 256, 0, st>>>(n, sel, gain, target, g->vw, wpart, incoming, best_id, cap, part, wnext,
                                      stats);
    SPX_LAUNCHED();
    g->ctr.launches += 4;
    unsigned long long hs[2] = {0, 0};
    SPX_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    ++rounds;
    moves += static_cast<int>(hs[0]);
    if (hs[0] == 0) break;
  }
  if (moves_out) *moves_out = moves;
  if (rounds_out) *rounds_out = rounds;
}

}  // namespace sphynx

using namespace sphynx;

extern "C" int sphynx_refine(sphynx_handle g, int32_t *part, int32_t K, double eps, int32_t max_rounds,
                             double *cut_out, double *imbalance_out, int32_t *moves_out, int32_t *rounds_out) {
  return guarded([&]() -> int {
    if (!g || !part) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (g->batch.count > 0) fail(SPHYNX_ERR_UNSUPPORTED, "refinement takes single graphs");
    int moves = 0, rounds = 0;
    refine_partition(g, part, K, eps, max_rounds, kRefineMaxDegree, &moves, &rounds);
    double cut = 0, cut2 = 0, imb = 0;
    eval_partition(g, part, K, &cut, &cut2, &imb);
    if (cut_out) *cut_out = cut;
    if (imbalance_out) *imbalance_out = imb;
    if (moves_out) *moves_out = moves;
    if (rounds_out) *rounds_out = rounds;
    return SPHYNX_OK;
  });
}
