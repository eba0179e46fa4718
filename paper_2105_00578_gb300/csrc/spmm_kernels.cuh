// spmm_kernels.cuh -- the Laplacian block product Y = L X without forming L.
//
// L is one of (Sec. 3.2, Eqs. 2-3, weighted rule):
//   combinatorial  (L_C X)_i = deg_i X_i - sum_j w_ij X_j
//   normalized     (L_N X)_i = X_i - s_i sum_j w_ij s_j X_j,   s = D^{-1/2}
// (the generalized problem applies L_C; its B = D is applied elsewhere).
//
// Schedules.  Rows with at most kShortDeg neighbours go to the short-row
// kernel: a warp owns 32 consecutive rows, stages their column indices (and
// weights) with coalesced loads into shared memory, and each lane then walks
// its own row, gathering X rows with 16-byte vector loads.  Longer rows are
// cut into work items of kLongChunk entries; a warp per item reduces its
// entries with shuffles into a partial row, and a finalise kernel adds the
// partials of each long row in a fixed order (deterministic results) and
// applies the epilogue.
//
// Epilogues.  Mode 0 stores L X.  Mode 1 is one step of the product-form
// polynomial preconditioner (Sec. 5.2): with t the input block,
//   t' = t - (L t) / theta_i   (stored in type TT),
//   y  = (first ? t / theta_i : y) + t' / theta_{i+1}.
#pragma once

#include "internal.cuh"

namespace sphynx {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 4;
constexpr int kStageCap = 32 * kShortDeg;

template <typename TI> struct AccOf { using T = float; };
template <> struct AccOf<double> { using T = double; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- row loads / stores (rows are 16-byte aligned for bp >= 4) --------------
template <int BP>
__device__ __forceinline__ void load_row(const double *__restrict__ p, double (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __ldg(p);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 2) {
      double2 v = __ldg(reinterpret_cast<const double2 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y;
    }
  }
}
template <int BP>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __ldg(p);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      float4 v = __ldg(reinterpret_cast<const float4 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  }
}
template <int BP>
__device__ __forceinline__ void load_row(const __nv_bfloat16 *__restrict__ p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __bfloat162float(p[0]);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      uint2 v = __ldg(reinterpret_cast<const uint2 *>(p + c));
      __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&v.x);
      __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&v.y);
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      o[c] = fa.x; o[c + 1] = fa.y; o[c + 2] = fb.x; o[c + 3] = fb.y;
    }
  }
}
// plain (coherent) loads for buffers written by the same launch sequence
template <int BP>
__device__ __forceinline__ void load_row_rw(const double *p, double (&o)[BP]) {
#pragma unroll
  for (int c = 0; c < BP; ++c) o[c] = p[c];
}
template <int BP>
__device__ __forceinline__ void load_row_rw(const float *p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = p[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      float4 v = *reinterpret_cast<const float4 *>(p + c);
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  }
}

template <int BP>
__device__ __forceinline__ void store_row(double *p, const double (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 2) *reinterpret_cast<double2 *>(p + c) = make_double2(v[c], v[c + 1]);
  }
}
template <int BP>
__device__ __forceinline__ void store_row(float *p, const float (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4)
      *reinterpret_cast<float4 *>(p + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
  }
}
// bf16 store rounds to nearest-even and returns the stored values in v
template <int BP>
__device__ __forceinline__ void store_row(__nv_bfloat16 *p, float (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = __float2bfloat16_rn(v[0]);
    v[0] = __bfloat162float(p[0]);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[c], v[c + 1]);
      __nv_bfloat162 b = __floats2bfloat162_rn(v[c + 2], v[c + 3]);
      uint2 u;
      u.x = *reinterpret_cast<unsigned *>(&a);
      u.y = *reinterpret_cast<unsigned *>(&b);
      *reinterpret_cast<uint2 *>(p + c) = u;
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      v[c] = fa.x; v[c + 1] = fa.y; v[c + 2] = fb.x; v[c + 3] = fb.y;
    }
  }
}

template <typename TA> __device__ __forceinline__ TA deg_of(const LapView &L, int64_t i);
template <> __device__ __forceinline__ double deg_of<double>(const LapView &L, int64_t i) { return L.deg[i]; }
template <> __device__ __forceinline__ float deg_of<float>(const LapView &L, int64_t i) { return L.degf[i]; }
template <typename TA> __device__ __forceinline__ TA dinv_of(const LapView &L, int64_t i);
template <> __device__ __forceinline__ double dinv_of<double>(const LapView &L, int64_t i) { return __ldg(L.dinv + i); }
template <> __device__ __forceinline__ float dinv_of<float>(const LapView &L, int64_t i) { return __ldg(L.dinvf + i); }

struct SpmmDev {              // kernel-side view of SpmmArgs
  const void *x;
  int ldx, ldy;
  void *y;
  void *tout;
  void *yacc;
  int first;
  const double *inv;
  int icur;
  const int *done;
};

// acc = sum_j w_ij (s_j) X_j of row `row`; epilogue applies the diagonal part.
template <int LAP, typename TI, typename TT, int BP, int MODE>
__device__ __forceinline__ void spmm_epilogue(const LapView &L, const SpmmDev &a, int64_t row,
                                              const typename AccOf<TI>::T (&acc)[BP]) {
  using TA = typename AccOf<TI>::T;
  const TI *x = static_cast<const TI *>(a.x);
  TA xi[BP];
  load_row<BP>(x + row * a.ldx, xi);
  TA out[BP];
  if constexpr (LAP == SPHYNX_NORMALIZED) {
    const TA s = dinv_of<TA>(L, row);
#pragma unroll
    for (int c = 0; c < BP; ++c) out[c] = xi[c] - s * acc[c];
  } else {
    const TA d = deg_of<TA>(L, row);
#pragma unroll
    for (int c = 0; c < BP; ++c) out[c] = d * xi[c] - acc[c];
  }
  if constexpr (MODE == 0) {
    store_row<BP>(static_cast<TA *>(a.y) + row * a.ldy, out);
  } else {
    const TA ic = static_cast<TA>(a.inv[a.icur]);
    const TA inx = static_cast<TA>(a.inv[a.icur + 1]);
    TA tn[BP];
#pragma unroll
    for (int c = 0; c < BP; ++c) tn[c] = xi[c] - out[c] * ic;
    store_row<BP>(static_cast<TT *>(a.tout) + row * a.ldx, tn);  // tn now holds the stored values
    TA *yp = static_cast<TA *>(a.yacc) + row * a.ldy;
    TA ya[BP];
    if (a.first) {
#pragma unroll
      for (int c = 0; c < BP; ++c) ya[c] = xi[c] * ic;
    } else {
      load_row_rw<BP>(yp, ya);
    }
#pragma unroll
    for (int c = 0; c < BP; ++c) ya[c] += tn[c] * inx;
    store_row<BP>(yp, ya);
  }
}

template <int LAP, typename TI, int BP, bool W>
__device__ __forceinline__ void spmm_accumulate(const LapView &L, const TI *__restrict__ x, int ldx,
                                                int j, float wv, typename AccOf<TI>::T (&acc)[BP]) {
  using TA = typename AccOf<TI>::T;
  TA xj[BP];
  load_row<BP>(x + static_cast<int64_t>(j) * ldx, xj);
  if constexpr (LAP == SPHYNX_NORMALIZED || W) {
    TA coef = W ? static_cast<TA>(wv) : TA(1);
    if constexpr (LAP == SPHYNX_NORMALIZED) coef *= dinv_of<TA>(L, j);
#pragma unroll
    for (int c = 0; c < BP; ++c) acc[c] += coef * xj[c];
  } else {
#pragma unroll
    for (int c = 0; c < BP; ++c) acc[c] += xj[c];
  }
}

template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_spmm_short(const LapView L, const SpmmDev a) {
  using TA = typename AccOf<TI>::T;
  __shared__ int s_col[kWarpsPerCta][kStageCap];
  __shared__ float s_w[kWarpsPerCta][W ? kStageCap : 1];
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = (static_cast<int64_t>(blockIdx.x) * kWarpsPerCta + wid) * 32;
  if (row0 >= L.n) return;  // uniform per warp
  const int64_t row = row0 + lane;
  const bool valid = row < L.n;
  int64_t rb = 0, re = 0;
  if (valid) {
    rb = L.rowptr[row];
    re = L.rowptr[row + 1];
  }
  const int nvalid = L.n - row0 < 32 ? static_cast<int>(L.n - row0) : 32;
  const int64_t wb = __shfl_sync(kFull, rb, 0);
  const int64_t we = __shfl_sync(kFull, re, nvalid - 1);
  const int64_t cnt = we - wb;
  const bool staged = cnt <= kStageCap;
  if (staged) {
    for (int e = lane; e < cnt; e += 32) {
      s_col[wid][e] = __ldg(L.col + wb + e);
      if constexpr (W) s_w[wid][e] = __ldg(L.w + wb + e);
    }
  }
  __syncwarp();
  if (!valid || re - rb > kShortDeg) return;
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  TA acc[BP];
#pragma unroll
  for (int c = 0; c < BP; ++c) acc[c] = TA(0);
  if (staged) {
    const int e0 = static_cast<int>(rb - wb), e1 = static_cast<int>(re - wb);
#pragma unroll 4
    for (int e = e0; e < e1; ++e)
      spmm_accumulate<LAP, TI, BP, W>(L, x, a.ldx, s_col[wid][e], W ? s_w[wid][e] : 0.f, acc);
  } else {
    for (int64_t e = rb; e < re; ++e)
      spmm_accumulate<LAP, TI, BP, W>(L, x, a.ldx, __ldg(L.col + e), W ? __ldg(L.w + e) : 0.f, acc);
  }
  spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, acc);
}

// One warp per long-row work item: partial[item] = sum over the item's entries.
template <int LAP, typename TI, int BP, bool W>
__global__ void __launch_bounds__(256)
k_spmm_long(const LapView L, const SpmmDev a, const int64_t *__restrict__ items, int64_t n_items,
            typename AccOf<TI>::T *__restrict__ partials) {
  using TA = typename AccOf<TI>::T;
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t item = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (item >= n_items) return;
  const int64_t b = items[item * 4 + 1], e = items[item * 4 + 2];
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  TA acc[BP];
#pragma unroll
  for (int c = 0; c < BP; ++c) acc[c] = TA(0);
  for (int64_t k = b + lane; k < e; k += 32)
    spmm_accumulate<LAP, TI, BP, W>(L, x, a.ldx, __ldg(L.col + k), W ? __ldg(L.w + k) : 0.f, acc);
#pragma unroll
  for (int c = 0; c < BP; ++c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(kFull, acc[c], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < BP; ++c) partials[item * BP + c] = acc[c];
  }
}

// One thread per long row: add its partials in item order, apply the epilogue.
template <int LAP, typename TI, typename TT, int BP, int MODE>
__global__ void __launch_bounds__(128)
k_spmm_finalize(const LapView L, const SpmmDev a, const int64_t *__restrict__ split, int64_t n_long,
                const typename AccOf<TI>::T *__restrict__ partials) {
  using TA = typename AccOf<TI>::T;
  if (a.done && *a.done) return;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_long) return;
  const int64_t row = split[t * 3], first = split[t * 3 + 1], cnt = split[t * 3 + 2];
  TA acc[BP];
#pragma unroll
  for (int c = 0; c < BP; ++c) acc[c] = TA(0);
  for (int64_t s = first; s < first + cnt; ++s) {
#pragma unroll
    for (int c = 0; c < BP; ++c) acc[c] += partials[s * BP + c];
  }
  spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, acc);
}

template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
void spmm_launch_t(sphynx_graph *g, const SpmmDev &a) {
  using TA = typename AccOf<TI>::T;
  const LapView L = g->view();
  cudaStream_t st = g->stream;
  const int64_t warps = (g->n + 31) / 32;
  const int64_t grid = (warps + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid > 0) {
    k_spmm_short<LAP, TI, TT, BP, W, MODE><<<static_cast<unsigned>(grid), 32 * kWarpsPerCta, 0, st>>>(L, a);
    SPX_LAUNCHED();
    g->ctr.launches++;
  }
  if (g->plan.n_long > 0) {
    TA *part = g->plan.partials.as<TA>();
    const int64_t gl = (g->plan.n_items * 32 + 255) / 256;
    k_spmm_long<LAP, TI, BP, W><<<static_cast<unsigned>(gl), 256, 0, st>>>(
        L, a, g->plan.items.as<int64_t>(), g->plan.n_items, part);
    SPX_LAUNCHED();
    const int64_t gf = (g->plan.n_long + 127) / 128;
    k_spmm_finalize<LAP, TI, TT, BP, MODE><<<static_cast<unsigned>(gf), 128, 0, st>>>(
        L, a, g->plan.split.as<int64_t>(), g->plan.n_long, part);
    SPX_LAUNCHED();
    g->ctr.launches += 2;
  }
}

template <int LAP, typename TI, typename TT, bool W, int MODE>
void spmm_bp(sphynx_graph *g, const SpmmDev &a, int bp) {
  switch (bp) {
    case 4: spmm_launch_t<LAP, TI, TT, 4, W, MODE>(g, a); break;
    case 8: spmm_launch_t<LAP, TI, TT, 8, W, MODE>(g, a); break;
    case 12: spmm_launch_t<LAP, TI, TT, 12, W, MODE>(g, a); break;
    case 16: spmm_launch_t<LAP, TI, TT, 16, W, MODE>(g, a); break;
    default: fail(SPHYNX_ERR_INVALID_ARG, "block width %d not supported", bp);
  }
}

template <typename TI, typename TT, int MODE>
void spmm_lapw(sphynx_graph *g, const SpmmDev &a, int lap, int bp) {
  const bool w = g->weighted;
  if (bp == 1) {
    if constexpr (MODE == 0 && !std::is_same<TI, __nv_bfloat16>::value) {
      if (lap == SPHYNX_NORMALIZED) {
        if (w) spmm_launch_t<SPHYNX_NORMALIZED, TI, TT, 1, true, 0>(g, a);
        else spmm_launch_t<SPHYNX_NORMALIZED, TI, TT, 1, false, 0>(g, a);
      } else {
        if (w) spmm_launch_t<SPHYNX_COMBINATORIAL, TI, TT, 1, true, 0>(g, a);
        else spmm_launch_t<SPHYNX_COMBINATORIAL, TI, TT, 1, false, 0>(g, a);
      }
      return;
    }
    fail(SPHYNX_ERR_INVALID_ARG, "single-column product only in plain mode for float/double");
  }
  if (lap == SPHYNX_NORMALIZED) {
    if (w) spmm_bp<SPHYNX_NORMALIZED, TI, TT, true, MODE>(g, a, bp);
    else spmm_bp<SPHYNX_NORMALIZED, TI, TT, false, MODE>(g, a, bp);
  } else {
    if (w) spmm_bp<SPHYNX_COMBINATORIAL, TI, TT, true, MODE>(g, a, bp);
    else spmm_bp<SPHYNX_COMBINATORIAL, TI, TT, false, MODE>(g, a, bp);
  }
}

void spmm_dispatch_f64(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);
void spmm_dispatch_f32(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);
void spmm_dispatch_bf16(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);

}  // namespace sphynx
